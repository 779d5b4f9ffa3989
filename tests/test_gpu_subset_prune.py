"""The estimate's subset distance (Eq. 1 on A_sel, B_sel, Algorithm 3) with
row pruning against the plain contraction and the oracle.

The pruned form contracts every subset row against the other subset's first
2,048 rows (upper bounds of NN distances), the first 2,048 rows of each
subset against the whole other subset (lower bounds of each directed
maximum), twice 1,024 of the rows whose upper bound reaches the current
bound against the whole other subset (a larger lower bound), and runs the
full contraction on the rows whose upper bound reaches the last bound. Its claim is equality with the plain
contraction in every field of the result, so each case runs the same
estimate both ways (the context's subset threshold set to 0 and to
infinity) and compares the decoded results field by field, then checks H
against the oracle's HD of the selected subsets."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_18207_gb300 import prohd
from paper_2511_18207_gb300 import workloads as W

from .gpu_util import ctx, dev, rel, torch_cuda

pytestmark = pytest.mark.gpu

FIELDS = ["H", "h_ab", "h_ba", "dir", "wit_a", "wit_b", "ab", "ba", "H_lowp", "n_rescored_a", "n_rescored_b",
          "status", "nsel_a", "nsel_b"]


def _both(A, B, **kw):
    torch_cuda()
    c = ctx()
    At, Bt = dev(A), dev(B)
    try:
        c.set_subset_prune_min_pairs(math.inf)
        plain = prohd.prohd_estimate_sync(At, Bt, want_indices=True, **kw)
        c.set_subset_prune_min_pairs(0.0)
        pruned = prohd.prohd_estimate_sync(At, Bt, want_indices=True, **kw)
    finally:
        c.set_subset_prune_min_pairs(1e9)
    for f in FIELDS:
        assert plain[f] == pruned[f], (f, plain[f], pruned[f])
    np.testing.assert_array_equal(plain["idxA"], pruned["idxA"])
    np.testing.assert_array_equal(plain["idxB"], pruned["idxB"])
    return pruned


def _oracle_check(A, B, r):
    sub = oracle.hausdorff(A[r["idxA"]], B[r["idxB"]])
    assert rel(r["H"], sub["H"]) <= 1e-5, (r["H"], sub["H"])


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_pruned_subset_hd_equals_plain_anisotropic_d256(prec):
    # the benchmark's law at 400k + 400k: subsets of about 15k rows per set
    A, B = W.anisotropic_pair(400_000, 400_000, 256, shift_sigma=0.1, t_frac=0.001, nu=3.0, seed=5)
    r = _both(A, B, m=8, alpha_c=0.01, precision=prec)
    assert r["status"] == "OK"
    assert min(r["nsel_a"], r["nsel_b"]) > 8192


@pytest.mark.parametrize("D,seed", [(64, 1), (128, 2), (100, 3)])
def test_pruned_subset_hd_equals_plain_mixtures(D, seed):
    # Gaussian mixtures (D = 100 pads the tiles' K dimension); subset bounds
    # of 9,600 rows per set admit the pruned form
    A, B = W.mixture_pair(120_000, D, 16, seed=seed)
    r = _both(A, B, m=8, alpha_c=0.02)
    assert r["status"] == "OK"
    _oracle_check(A, B, r)


def test_pruned_subset_hd_uneven_sets():
    # one subset about twice the other
    A, B = W.mixture_pair(150_000, 64, 8, seed=9)
    B = B[:70_000]
    r = _both(A, B, m=8, alpha_c=0.03)
    assert r["nsel_a"] > 1.5 * r["nsel_b"]
    _oracle_check(A, B, r)


def test_pruned_subset_hd_far_outlier_and_duplicates():
    # a single far point decides H; many duplicated rows tie for minima
    rng = np.random.default_rng(4)
    A = rng.standard_normal((120_000, 64)).astype(np.float32)
    B = rng.standard_normal((120_000, 64)).astype(np.float32)
    A[77_777] += np.float32(40.0)
    B[:30_000] = B[30_000:60_000]
    r = _both(A, B, m=6, alpha_c=0.03)
    _oracle_check(A, B, r)
    assert r["wit_a"] == 77_777


def test_subset_prune_threshold_rejects_negative():
    c = ctx()
    with pytest.raises(prohd.ProHDError):
        c.set_subset_prune_min_pairs(-1.0)
