"""ProHD end to end (Algorithm 3) on the GPU against the oracle.

Contract: the GPU's candidate sets equal the oracle's selection for the GPU's
own directions (bit-exact), H_hat equals the oracle's exact HD of those
subsets (relative 1e-5), and the directions agree with the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2511_18207_gb300 import prohd
from paper_2511_18207_gb300 import workloads as W

from .gpu_util import dev, prune_always, rel, torch_cuda  # noqa: F401 (fixture)

pytestmark = pytest.mark.gpu


def _run(A, B, m, alpha, prec="fp16", alpha_p=None):
    torch_cuda()
    r = prohd.prohd_estimate_sync(dev(A), dev(B), want_indices=True, want_dirs=True, m=m, alpha_c=alpha,
                                  alpha_p=alpha_p, precision=prec)
    assert r["status"] == "OK", r
    dirs = r["dirs"]
    ap = alpha / max(m, 1) if alpha_p is None else alpha_p
    kA = oracle.k_list(A.shape[0], 1 + m, alpha, ap)
    kB = oracle.k_list(B.shape[0], 1 + m, alpha, ap)
    ia, ib = oracle.select(A, dirs, kA), oracle.select(B, dirs, kB)
    np.testing.assert_array_equal(r["idxA"], ia)
    np.testing.assert_array_equal(r["idxB"], ib)
    assert r["nsel_a"] == ia.size and r["nsel_b"] == ib.size
    sub = oracle.hausdorff(A[ia], B[ib])
    assert rel(r["H"], sub["H"]) <= 1e-5, (r["H"], sub["H"])
    # witnesses are indices into the full sets
    d = np.sqrt(((A[r["wit_a"]].astype(np.float64) - B[r["wit_b"]]) ** 2).sum())
    assert d == pytest.approx(r["H"], rel=1e-12)
    return r


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
def test_estimate_config_small(prec):
    # N(0,I16) vs N(0.5,I16) with 1% outliers; centroid + top-2 PCs; 2% per side
    A, B = W.gaussian_outliers(2000, 2000, 16, seed=0)
    r = _run(A, B, m=2, alpha=0.02, prec=prec, alpha_p=0.02)
    o = oracle.prohd(A, B, alpha=0.02, m=2, alpha_p=0.02, seed=0)
    # end to end against the oracle's own directions: same candidate sets here
    np.testing.assert_array_equal(r["idxA"], o["idxA"])
    np.testing.assert_array_equal(r["idxB"], o["idxB"])
    assert rel(r["H"], o["H_hat"]) <= 1e-5


def test_estimate_defaults_random_clouds():
    A, B = W.random_clouds(20_000, 15_000, 8, seed=2)
    _run(A, B, m=2, alpha=0.01)


def test_estimate_mixture_d256():
    A, B = W.mixture_pair(20_000, 256, 16, seed=1)
    _run(A, B, m=8, alpha=0.01)


def test_estimate_host_entry_matches_device():
    torch = torch_cuda()
    A, B = W.gaussian_outliers(3000, 2500, 16, seed=3)
    c = prohd.context()
    p = prohd.default_params(m=2, alpha_c=0.02)
    res = c.prohd_estimate_host(torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory(), params=p)
    torch.cuda.current_stream().synchronize()
    h = prohd.decode_result(res)
    d = prohd.prohd_estimate_sync(dev(A), dev(B), m=2, alpha_c=0.02)
    assert h["H"] == d["H"] and h["nsel_a"] == d["nsel_a"] and h["nsel_b"] == d["nsel_b"]


def test_estimate_host_entry_with_row_range_copies():
    # both sets of at least 131,072 rows: the host entry copies each set in
    # two row ranges on its own stream and the Gram reads each range as it
    # lands (four launches whose partials are summed together); the estimate
    # matches the device entry's, here to the bit
    torch = torch_cuda()
    A, B = W.anisotropic_pair(140_000, 150_000, 64, shift_sigma=0.1, t_frac=0.001, nu=3.0, seed=8)
    c = prohd.context()
    p = prohd.default_params(m=8, alpha_c=0.01)
    for _ in range(2):  # the second call reuses the context's copy stream and events
        res = c.prohd_estimate_host(torch.from_numpy(A).pin_memory(), torch.from_numpy(B).pin_memory(), params=p)
        torch.cuda.current_stream().synchronize()
        h = prohd.decode_result(res)
        d = prohd.prohd_estimate_sync(dev(A), dev(B), m=8, alpha_c=0.01)
        assert h["status"] == "OK"
        assert h["H"] == d["H"] and h["nsel_a"] == d["nsel_a"] and h["nsel_b"] == d["nsel_b"], (h, d)


@pytest.mark.parametrize("D", [64, 256, 13])
@pytest.mark.parametrize("where", ["A_first", "A_middle", "A_last", "B_last_inf"])
def test_estimate_nonfinite_input_is_reported(D, where):
    # The covariance pass reads every point, so a non-finite coordinate
    # anywhere (first chunk, middle, the ragged last chunk of a set) must
    # surface as ENONFINITE; D = 13 takes the CUDA-core covariance kernel.
    torch_cuda()
    A, B = W.anisotropic_pair(30_001, 20_003, D, seed=3)
    if where == "A_first":
        A[0, D - 1] = np.nan
    elif where == "A_middle":
        A[17_777, D // 2] = np.nan
    elif where == "A_last":
        A[-1, 0] = np.nan
    else:
        B[-1, D - 1] = np.inf
    r = prohd.prohd_estimate_sync(dev(A), dev(B), m=2, alpha_c=0.01)
    assert r["status"] == "ENONFINITE", r["status"]


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
@pytest.mark.parametrize("shape", [(6_001, 5_003, 16, 2, 0.02), (20_000, 17_771, 256, 8, 0.01),
                                   # other set above 32,768 rows, subsets above 1,024: the row-pruned passes
                                   (60_000, 50_001, 32, 3, 0.02)])
def test_estimate_refined_matches_oracle(prec, shape, prune_always):
    # params.refine = 1: max(h(A_sel, B), h(B_sel, A)) with each selected
    # point's nearest neighbour searched in the whole other set; never above H
    torch_cuda()
    nA, nB, D, m, alpha = shape
    if D == 16:
        A, B = W.gaussian_outliers(nA, nB, D, seed=5)
    else:
        A, _ = W.mixture_pair(nA, D, 16, seed=6)
        _, B = W.mixture_pair(nB, D, 16, seed=7)
    r0 = prohd.prohd_estimate_sync(dev(A), dev(B), want_indices=True, m=m, alpha_c=alpha, precision=prec)
    r = prohd.prohd_estimate_sync(dev(A), dev(B), want_indices=True, m=m, alpha_c=alpha, precision=prec, refine=1)
    assert r["status"] == "OK", r
    # same candidate sets as the plain estimate
    np.testing.assert_array_equal(r["idxA"], r0["idxA"])
    np.testing.assert_array_equal(r["idxB"], r0["idxB"])
    o = oracle.refined(A, B, r["idxA"], r["idxB"])
    assert rel(r["h_ab"], o["h_ab"]) <= 1e-5, (r["h_ab"], o["h_ab"])
    assert rel(r["h_ba"], o["h_ba"]) <= 1e-5, (r["h_ba"], o["h_ba"])
    assert rel(r["H"], o["H1"]) <= 1e-5
    assert r["dir"] == (0 if r["h_ab"] >= r["h_ba"] else 1)
    # the witness is a selected point and its nearest neighbour in the full set
    sel = r["idxA"] if r["dir"] == 0 else r["idxB"]
    assert (r["wit_a"] if r["dir"] == 0 else r["wit_b"]) in set(sel.tolist())
    d = np.sqrt(((A[r["wit_a"]].astype(np.float64) - B[r["wit_b"]]) ** 2).sum())
    assert d == pytest.approx(r["H"], rel=1e-12)
    if D == 16:
        assert r["H"] <= oracle.hausdorff(A, B)["H"] * (1 + 1e-7)


def test_estimate_refined_with_given_directions():
    torch = torch_cuda()
    A, B = W.mixture_pair(12_000, 64, 8, seed=8)
    rng = np.random.default_rng(9)
    dirs = rng.standard_normal((5, 64))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    kA, kB = [90] + [20] * 4, [70] + [15] * 4
    c = prohd.context()
    idxA = torch.empty(A.shape[0], dtype=torch.int32, device="cuda")
    idxB = torch.empty(B.shape[0], dtype=torch.int32, device="cuda")
    out = c.prohd_estimate_dirs(dev(A), dev(B), torch.from_numpy(dirs).cuda(), kA, kB, precision="fp16",
                                idxA=idxA, idxB=idxB, refine=1)
    torch.cuda.synchronize()
    r = prohd.decode_result(out)
    assert r["status"] == "OK"
    ia, ib = oracle.select(A, dirs, kA), oracle.select(B, dirs, kB)
    np.testing.assert_array_equal(idxA[: r["nsel_a"]].cpu().numpy(), ia)
    o = oracle.refined(A, B, ia, ib)
    assert rel(r["H"], o["H1"]) <= 1e-5


def test_refine_must_be_zero_or_one():
    torch_cuda()
    A, B = W.random_clouds(500, 400, 8, seed=1)
    with pytest.raises(prohd.ProHDError):
        prohd.prohd_estimate_sync(dev(A), dev(B), refine=2)


def _adaptive(A, B, alpha, alpha_max, tol, m, prec):
    torch = torch_cuda()
    D = A.shape[1]
    dirs = torch.empty((1 + m, D), dtype=torch.float64, device="cuda")
    idxA = torch.empty(A.shape[0], dtype=torch.int32, device="cuda")
    idxB = torch.empty(B.shape[0], dtype=torch.int32, device="cuda")
    out, sched = prohd.context().prohd_estimate_adaptive(dev(A), dev(B), alpha_max, tol, m=m, alpha_c=alpha,
                                                         precision=prec, idxA=idxA, idxB=idxB, dirs=dirs)
    torch.cuda.synchronize()
    r = prohd.decode_result(out)
    assert r["status"] == "OK", r
    d = dirs.cpu().numpy()
    o = oracle.adaptive(A, B, alpha, alpha_max, tol, dirs=d)
    assert sched["steps"] == o["steps"] and sched["reason"] == o["reason"], (sched, o["H"], o["reason"])
    assert sched["nsel_a"] == o["nsel_a"] and sched["nsel_b"] == o["nsel_b"]
    np.testing.assert_allclose(sched["H"], o["H"], rtol=1e-5)
    assert sched["alpha_c"] == o["alpha"] and sched["alpha_p"] == pytest.approx(o["alpha_p"], rel=1e-15)
    np.testing.assert_array_equal(idxA[: r["nsel_a"]].cpu().numpy(), o["idxA"])
    np.testing.assert_array_equal(idxB[: r["nsel_b"]].cpu().numpy(), o["idxB"])
    assert r["H"] == sched["H"][-1]
    # never decreasing along the schedule
    assert all(b >= a for a, b in zip(sched["H"], sched["H"][1:]))
    return r, sched, o


@pytest.mark.parametrize("prec", ["fp16", "fp32"])
def test_adaptive_alpha_matches_oracle(prec):
    # N(0,I16) vs N(0.5,I16) with outliers; doubling 0.5% -> at most 32%
    A, B = W.gaussian_outliers(6_001, 5_003, 16, seed=11)
    _adaptive(A, B, 0.005, 0.3, 0.0, 2, prec)


def test_adaptive_alpha_stable_stop_d64():
    A, _ = W.mixture_pair(20_000, 64, 8, seed=12)
    _, B = W.mixture_pair(17_771, 64, 8, seed=13)
    r, sched, _ = _adaptive(A, B, 0.0025, 0.05, 0.01, 4, "bf16")
    assert sched["reason"] in ("stable", "budget")


def test_adaptive_alpha_reaches_the_exact_hd():
    # alpha 1% doubled up to 64% keeps every point (k >= n/2 per side): H
    A, B = W.random_clouds(4_000, 3_001, 8, seed=14)
    r, sched, _ = _adaptive(A, B, 0.01, 0.99, 0.0, 2, "fp16")
    if sched["reason"] == "all":
        assert rel(r["H"], oracle.hausdorff(A, B)["H"]) <= 1e-5
    assert r["H"] <= oracle.hausdorff(A, B)["H"] * (1 + 1e-7)


def test_adaptive_alpha_single_step_and_bad_arguments():
    torch = torch_cuda()
    A, B = W.random_clouds(2_000, 1_500, 4, seed=15)
    out, sched = prohd.context().prohd_estimate_adaptive(dev(A), dev(B), 0.02, 0.0, m=1, alpha_c=0.02)
    torch.cuda.synchronize()
    assert sched["steps"] == 1 and sched["reason"] == "budget"
    r = prohd.decode_result(out)
    r1 = prohd.prohd_estimate_sync(dev(A), dev(B), m=1, alpha_c=0.02, refine=1)
    assert r["H"] == r1["H"] and r["nsel_a"] == r1["nsel_a"]
    with pytest.raises(prohd.ProHDError):
        prohd.context().prohd_estimate_adaptive(dev(A), dev(B), 0.01, 0.0, m=1, alpha_c=0.02)
    with pytest.raises(prohd.ProHDError):
        prohd.context().prohd_estimate_adaptive(dev(A), dev(B), 0.5, -1.0, m=1, alpha_c=0.02)


def test_adaptive_alpha_with_pruned_refinement(prune_always):
    # sets above 32,768 rows: every step's refinement takes the row-pruned passes
    A, B = W.gaussian_outliers(40_001, 36_003, 16, seed=16)
    _adaptive(A, B, 0.005, 0.08, 0.0, 2, "fp16")


def test_refined_with_every_point_selected_is_the_exact_hd():
    # 2k >= n on every direction: both subsets are the whole sets, so the
    # refined estimate is H itself
    A, B = W.random_clouds(700, 600, 8, seed=17)
    r = prohd.prohd_estimate_sync(dev(A), dev(B), m=2, alpha_c=0.6, alpha_p=0.6, refine=1)
    assert r["status"] == "OK" and r["nsel_a"] == 700 and r["nsel_b"] == 600
    assert rel(r["H"], oracle.hausdorff(A, B)["H"]) <= 1e-5


def test_adaptive_alpha_single_step_budget_edge():
    # alpha_max just below the second step: one step, stop reason "budget"
    torch = torch_cuda()
    A, B = W.gaussian_outliers(3_000, 2_500, 16, seed=18)
    out, sched = prohd.context().prohd_estimate_adaptive(dev(A), dev(B), 0.02 * 2 - 1e-12, 0.0, m=2, alpha_c=0.02)
    torch.cuda.synchronize()
    assert sched["steps"] == 1 and sched["reason"] == "budget"
    o = oracle.adaptive(A, B, 0.02, 0.04 - 1e-12, 0.0, dirs=None, m=2)
    assert o["steps"] == 1 and o["reason"] == "budget"
