"""GPU exact Hausdorff distance (Eq. 1) against the FP64 oracle.

Tolerances: FP32 path and the tensor paths after rescoring agree with the FP64
oracle to relative 1e-5 (FP32 rounding of the distances that choose the
witness; the witness distance itself is FP64). Before rescoring, the
low-precision estimate H_lowp agrees to 2e-3 (BF16) / 5e-4 (FP16)."""
import numpy as np
import pytest

import oracle
from paper_2511_18207_gb300 import prohd
from paper_2511_18207_gb300 import workloads as W

from .gpu_util import ctx, dev, prune_always, rel, torch_cuda  # noqa: F401 (fixture)

pytestmark = pytest.mark.gpu

PRECS = ["fp32", "fp16", "bf16"]


def _check(A, B, prec, tol=1e-5):
    torch_cuda()
    ref = oracle.hausdorff(A, B)
    r = prohd.hausdorff_exact_sync(dev(A), dev(B), prec)
    assert r["status"] == "OK", r
    assert rel(r["H"], ref["H"]) <= tol or abs(r["H"] - ref["H"]) <= 1e-6, (prec, r["H"], ref["H"])
    assert rel(r["h_ab"], ref["h_ab"]) <= tol or abs(r["h_ab"] - ref["h_ab"]) <= 1e-6
    assert rel(r["h_ba"], ref["h_ba"]) <= tol or abs(r["h_ba"] - ref["h_ba"]) <= 1e-6
    # the witnesses are valid: their FP64 distance is the reported value
    ia, jb = r["ab"]
    d = np.sqrt(((A[ia].astype(np.float64) - B[jb]) ** 2).sum())
    assert d == pytest.approx(r["h_ab"], rel=1e-12, abs=1e-12)
    jb2, ia2 = r["ba"]
    d = np.sqrt(((B[jb2].astype(np.float64) - A[ia2]) ** 2).sum())
    assert d == pytest.approx(r["h_ba"], rel=1e-12, abs=1e-12)
    return r, ref


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("nA,nB,D", [(1, 1, 3), (1, 7, 16), (9, 1, 16), (300, 517, 16), (1000, 777, 64),
                                     (700, 1300, 100), (513, 257, 256), (129, 255, 13), (2000, 2000, 16)])
def test_hd_parity(prec, nA, nB, D):
    rng = np.random.default_rng(nA * 31 + nB * 7 + D)
    A = rng.standard_normal((nA, D)).astype(np.float32)
    B = (rng.standard_normal((nB, D)) * 1.3 + 0.2).astype(np.float32)
    _check(A, B, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_hd_config_small(prec):
    A, B = W.gaussian_outliers(2000, 2000, 16, seed=0)
    r, ref = _check(A, B, prec)
    if prec != "fp32":
        lim = 2e-3 if prec == "bf16" else 5e-4
        assert rel(r["H_lowp"], ref["H"]) <= lim, (r["H_lowp"], ref["H"])
        assert r["n_rescored_a"] >= 1 and r["n_rescored_b"] >= 1


@pytest.mark.parametrize("prec", PRECS)
def test_hd_identical_and_duplicates(prec):
    torch_cuda()
    rng = np.random.default_rng(5)
    A = rng.standard_normal((400, 32)).astype(np.float32)
    r = prohd.hausdorff_exact_sync(dev(A), dev(A), prec)
    assert r["H"] == 0.0 and r["status"] == "OK"
    # many duplicate points and a far outlier
    B = np.repeat(A[:10], 50, axis=0)
    B[123] += 40.0
    _check(A, B, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_hd_offset_data(prec):
    # far from the origin: centring inside the tensor path keeps precision
    rng = np.random.default_rng(9)
    A = (rng.standard_normal((600, 48)) + 1000.0).astype(np.float32)
    B = (rng.standard_normal((500, 48)) * 0.5 + 1000.5).astype(np.float32)
    _check(A, B, prec)


def test_hd_nonfinite_is_reported():
    torch_cuda()
    A = np.zeros((64, 8), dtype=np.float32)
    B = np.ones((64, 8), dtype=np.float32)
    A[3, 2] = np.nan
    for prec in ("fp16", "bf16"):
        r = prohd.hausdorff_exact_sync(dev(A), dev(B), prec)
        assert r["status"] == "ENONFINITE"


def test_hd_invalid_arguments():
    torch_cuda()
    c = ctx()
    A = dev(np.zeros((4, 300), dtype=np.float32))
    with pytest.raises(prohd.ProHDError, match="ENOTSUP"):
        c.hausdorff_exact(A, A, "fp16")


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_hd_lowp_rows_within_margin(prec):
    # the low-precision row minima must lie inside the interval the rescoring
    # logic assumes: checked through the final answer on data whose nearest
    # neighbour distances are nearly equal (many candidates)
    rng = np.random.default_rng(21)
    A = rng.standard_normal((1500, 128)).astype(np.float32)
    B = rng.standard_normal((1400, 128)).astype(np.float32)
    _check(A, B, prec)


def _pruned(A, B, prec="fp16"):
    torch = torch_cuda()
    out, kept = ctx().hausdorff_exact_pruned(dev(A), dev(B), prec, want_kept=True)
    torch.cuda.synchronize()
    return prohd.decode_hd(out), kept


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_hd_pruned_matches_oracle(prec, prune_always):
    # both sets above the pruning threshold (32,768 rows); ragged sizes
    A, B = W.gaussian_outliers(40_001, 36_003, 16, seed=21)
    r, kept = _pruned(A, B, prec)
    assert r["status"] == "OK", r
    assert 0 < kept[0] <= A.shape[0] and 0 < kept[1] <= B.shape[0]
    o = oracle.hausdorff(A, B)
    assert rel(r["H"], o["H"]) <= 1e-5 and rel(r["h_ab"], o["h_ab"]) <= 1e-5 and rel(r["h_ba"], o["h_ba"]) <= 1e-5
    d = np.sqrt(((A[r["wit_a"]].astype(np.float64) - B[r["wit_b"]]) ** 2).sum())
    assert d == pytest.approx(r["H"], rel=1e-12)


@pytest.mark.parametrize("D", [64, 256])
def test_hd_pruned_equals_the_dense_path(D, prune_always):
    # a mixture pair with heavy-tailed points: most rows are dropped, the
    # result is the plain contraction's
    torch = torch_cuda()
    A = W.student_t_mixture(150_000, D, K=8, nu=3.0, seed=22)
    B = W.student_t_mixture(120_001, D, K=8, nu=3.0, seed=23)
    r, kept = _pruned(A, B)
    dense = prohd.decode_hd(ctx().hausdorff_exact(dev(A), dev(B), "fp16"))
    torch.cuda.synchronize()
    assert r["status"] == "OK" and dense["status"] == "OK"
    # both are the FP32 path's result; only the FP32 argmin of a row within
    # rounding of the maximum could tell them apart
    assert rel(r["H"], dense["H"]) <= 1e-6 and rel(r["h_ab"], dense["h_ab"]) <= 1e-6
    assert rel(r["h_ba"], dense["h_ba"]) <= 1e-6
    assert kept[0] < A.shape[0] and kept[1] < B.shape[0]
    # the witness rows are real nearest-neighbour pairs at distance H
    d = np.sqrt(((A[r["wit_a"]].astype(np.float64) - B[r["wit_b"]]) ** 2).sum())
    assert d == pytest.approx(r["H"], rel=1e-12)


def test_hd_pruned_small_sets_take_the_plain_path():
    A, B = W.random_clouds(5_000, 40_000, 8, seed=24)
    r, kept = _pruned(A, B)
    assert kept == [-1, -1]
    assert rel(r["H"], oracle.hausdorff(A, B)["H"]) <= 1e-5


def test_hd_pruned_below_the_pair_threshold_takes_the_plain_path():
    # 40,001 x 36,003 pairs are below the default threshold (4e9)
    A, B = W.gaussian_outliers(40_001, 36_003, 16, seed=25)
    r, kept = _pruned(A, B)
    assert kept == [-1, -1]
    assert rel(r["H"], oracle.hausdorff(A, B)["H"]) <= 1e-5


def test_hd_pruned_identical_sets(prune_always):
    # H = 0: the lower bounds are 0, nothing is dropped, the result is exact
    A = W.student_t_mixture(40_000, 32, K=4, nu=3.0, seed=26)
    r, kept = _pruned(A, A.copy())
    assert r["status"] == "OK" and r["H"] == 0.0
    assert kept == [A.shape[0], A.shape[0]]


def test_hd_pruned_with_duplicated_rows(prune_always):
    # repeated rows (ties in every minimum) in both sets
    rng = np.random.default_rng(27)
    base = W.student_t_mixture(20_000, 32, K=4, nu=3.0, seed=27)
    A = np.concatenate([base, base[rng.integers(0, 20_000, 20_000)]])
    B = np.concatenate([base[:18_000] + 0.05, base[rng.integers(0, 20_000, 18_000)]]).astype(np.float32)
    r, kept = _pruned(A, B)
    dense = prohd.decode_hd(ctx().hausdorff_exact(dev(A), dev(B), "fp16"))
    assert r["status"] == "OK" and rel(r["H"], dense["H"]) <= 1e-6
    assert rel(r["H"], oracle.hausdorff(A, B)["H"]) <= 1e-5
