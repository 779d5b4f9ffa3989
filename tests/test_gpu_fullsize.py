"""Parity at full size, in the configuration the benchmark times.

Two workloads:
- the 2M x 2M x 256 anisotropic pair: centroid axis plus 8 components,
  alpha = 0.01 per side, FP16 tiles (and BF16);
- the 200k x 200k x 256 mixture pair, with BF16 tiles.

The oracle cannot redo the whole computation at these sizes in a test, so
the outputs it can compute one by one are compared exactly:
- the candidate sets, bit-exact, for the GPU's own directions (the oracle's
  full FP64 selection);
- the centroid axis;
- the nearest-neighbour distance of each witness row, recomputed in FP64;
- a sample of rows, whose distances must not exceed the reported maximum.
At 200k the subset HD is small enough for the oracle's full computation."""
import numpy as np
import pytest

import oracle
from paper_2511_18207_gb300 import prohd
from paper_2511_18207_gb300 import workloads as W

from .gpu_util import ctx, dev, rel, torch_cuda
from .test_gpu_directions import _angle, _axis_bound

pytestmark = pytest.mark.gpu

M_PCS, ALPHA = 8, 0.01


@pytest.fixture(scope="module")
def pair_2m():
    torch_cuda()
    return W.anisotropic_pair(2_000_000, 2_000_000, 256, shift_sigma=0.1, t_frac=0.001, nu=3.0, seed=0)


def _estimate(At, Bt, prec):
    return prohd.prohd_estimate_sync(At, Bt, want_indices=True, want_dirs=True, m=M_PCS, alpha_c=ALPHA,
                                     precision=prec)


def _row_nn(X, Y, i):
    """FP64 nearest-neighbour distance of row i of X in Y (the oracle)."""
    return oracle.directed_hd(X, Y, i, i + 1)[0]


def _check_witnesses(A, B, r, ia, ib, nsample, seed):
    """The witness rows of h_ab and h_ba attain them; sampled rows stay below."""
    As, Bs = A[ia], B[ib]
    wa = int(np.searchsorted(ia, r["ab"][0]))
    wb = int(np.searchsorted(ib, r["ba"][0]))
    assert ia[wa] == r["ab"][0] and ib[wb] == r["ba"][0]
    assert rel(_row_nn(As, Bs, wa), r["h_ab"]) <= 1e-5
    assert rel(_row_nn(Bs, As, wb), r["h_ba"]) <= 1e-5
    rng = np.random.default_rng(seed)
    for i in rng.choice(len(ia), size=nsample, replace=False):
        assert _row_nn(As, Bs, int(i)) <= r["h_ab"] * (1 + 1e-5)
    for i in rng.choice(len(ib), size=nsample, replace=False):
        assert _row_nn(Bs, As, int(i)) <= r["h_ba"] * (1 + 1e-5)


def test_full_size_2m_estimate_matches_oracle(pair_2m):
    A, B = pair_2m
    At, Bt = dev(A), dev(B)
    r = _estimate(At, Bt, "fp16")
    assert r["status"] == "OK", r
    dirs = r["dirs"]
    # selection: bit-exact against the oracle's full FP64 selection for these directions
    kA = oracle.k_list(A.shape[0], 1 + M_PCS, ALPHA, ALPHA / M_PCS)
    kB = oracle.k_list(B.shape[0], 1 + M_PCS, ALPHA, ALPHA / M_PCS)
    ia, ib = oracle.select(A, dirs, kA), oracle.select(B, dirs, kB)
    np.testing.assert_array_equal(r["idxA"], ia)
    np.testing.assert_array_equal(r["idxB"], ib)
    # centroid axis against the FP64 centroids
    axis = oracle.centroid_axis(oracle.centroid(A), oracle.centroid(B))
    assert _angle(dirs[0], axis) <= _axis_bound(A, B)
    # the components are unit vectors, orthogonal to each other
    G = dirs[1:] @ dirs[1:].T
    assert np.abs(G - np.eye(M_PCS)).max() <= 1e-9
    # subset HD: witnesses and a sample of rows, in FP64
    _check_witnesses(A, B, r, ia, ib, nsample=32, seed=1)
    # BF16 tiles: same candidates, same FP32-rescored result
    rb = _estimate(At, Bt, "bf16")
    assert rb["status"] == "OK"
    np.testing.assert_array_equal(rb["idxA"], ia)
    assert rel(rb["H"], r["H"]) <= 1e-5


def test_full_size_2m_exact_hd_witness(pair_2m):
    # the exact HD of the full sets (row-pruned form, equal to the dense
    # one): the witness rows attain h_ab and h_ba over the whole other set
    A, B = pair_2m
    torch = torch_cuda()
    out = ctx().hausdorff_exact_pruned(dev(A), dev(B), "fp16")
    torch.cuda.synchronize()
    r = prohd.decode_hd(out)
    assert r["status"] == "OK", r
    assert rel(_row_nn(A, B, int(r["ab"][0])), r["h_ab"]) <= 1e-5
    assert rel(_row_nn(B, A, int(r["ba"][0])), r["h_ba"]) <= 1e-5
    rng = np.random.default_rng(2)
    for i in rng.choice(A.shape[0], size=4, replace=False):
        assert _row_nn(A, B, int(i)) <= r["h_ab"] * (1 + 1e-5)
    assert r["H"] == max(r["h_ab"], r["h_ba"])


def test_full_size_200k_mixture_bf16():
    # 16-component mixtures, BF16 tiles: the subset HD in full against the oracle
    torch = torch_cuda()
    A, B = W.mixture_pair(200_000, 256, 16, seed=0)
    At, Bt = dev(A), dev(B)
    r = _estimate(At, Bt, "bf16")
    assert r["status"] == "OK", r
    dirs = r["dirs"]
    kA = oracle.k_list(A.shape[0], 1 + M_PCS, ALPHA, ALPHA / M_PCS)
    kB = oracle.k_list(B.shape[0], 1 + M_PCS, ALPHA, ALPHA / M_PCS)
    ia, ib = oracle.select(A, dirs, kA), oracle.select(B, dirs, kB)
    np.testing.assert_array_equal(r["idxA"], ia)
    np.testing.assert_array_equal(r["idxB"], ib)
    sub = oracle.hausdorff(A[ia], B[ib])
    assert rel(r["H"], sub["H"]) <= 1e-5
    assert rel(r["h_ab"], sub["h_ab"]) <= 1e-5 and rel(r["h_ba"], sub["h_ba"]) <= 1e-5
    # the exact HD of the full sets: witnesses attain it
    ex = prohd.decode_hd(ctx().hausdorff_exact(At, Bt, "bf16"))
    torch.cuda.synchronize()
    assert ex["status"] == "OK"
    assert rel(_row_nn(A, B, int(ex["ab"][0])), ex["h_ab"]) <= 1e-5
    assert rel(_row_nn(B, A, int(ex["ba"][0])), ex["h_ba"]) <= 1e-5
