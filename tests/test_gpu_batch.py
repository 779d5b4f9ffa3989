"""Batched ProHD (many independent pairs in one planned, graph-captured run)
against the FP64 oracle, pair by pair.

Per pair the contract is the single-pair one: the candidate sets equal the
oracle's selection for the GPU's own directions (bit-exact), H_hat equals the
oracle's exact HD of those subsets (relative 1e-5; the batch runs the FP32
direct-difference subset HD), the witnesses are indices into the pair's own
sets, and the directions agree with the definition: centroid axis to the
oracle's within the FP32 partial-sum bound, eigenvalues to the oracle's and
to the exact spectrum within 1.5e-5 lambda_1 (a Ritz value's error is at most
its residual plus the covariance perturbation), and each component's angle
to the exact eigenvector of the oracle's FP64 covariance wherever its
eigengap makes the angle well defined (residual 2e-6 lambda_1 and covariance
perturbation 1e-5 lambda_1 over the gap)."""
import numpy as np
import pytest

import oracle
from paper_2511_18207_gb300 import prohd
from paper_2511_18207_gb300 import workloads as W

from .gpu_util import ctx, dev, rel, torch_cuda

pytestmark = pytest.mark.gpu

# (nA, nB, D): every D class, ragged tails, a one-point set, sets much larger
# than one Gram item, D not a power of two
SPEC = [(1000, 1000, 64), (2500, 1200, 128), (7001, 3333, 256), (40_000, 9000, 64), (4097, 4096, 128),
        (1, 5, 64), (300, 20_000, 256), (65_537, 1000, 128), (5000, 5003, 192), (2000, 3000, 8),
        (33_333, 31_000, 256), (1500, 60_000, 96)]


def _pairs(spec, seed=0):
    out = []
    for i, (na, nb, D) in enumerate(spec):
        K = 4 + (i * 7) % 29
        out.append((W.gaussian_mixture(na, D, K, seed=2 * (seed + i)),
                    W.gaussian_mixture(nb, D, K, seed=2 * (seed + i) + 1)))
    return out


def _angle(u, v):
    c = abs(float(np.dot(u, v)) / (np.linalg.norm(u) * np.linalg.norm(v)))
    return float(np.arccos(min(c, 1.0)))


def _run(pairs, m=8, alpha=0.01, graph=True, tune=None, precision="fp16"):
    torch = torch_cuda()
    dpairs = [(dev(A), dev(B)) for A, B in pairs]
    b = prohd.Batch(ctx(), dpairs, m=m, alpha_c=alpha, precision=precision)
    b.use_graph(graph)
    if tune is not None:
        b.set_tunables(*tune)
    b.run()
    torch.cuda.synchronize()
    return b, b.results()


def _check_pair(b, i, A, B, r, m, alpha, check_dirs=True):
    assert r["status"] == "OK", (i, r["status"])
    ap = alpha / m
    nd = 1 + m
    dirs, ia, ib = b.pair_outputs(i, r["nsel_a"], r["nsel_b"])
    kA = oracle.k_list(A.shape[0], nd, alpha, ap)
    kB = oracle.k_list(B.shape[0], nd, alpha, ap)
    np.testing.assert_array_equal(ia, oracle.select(A, dirs, kA))
    np.testing.assert_array_equal(ib, oracle.select(B, dirs, kB))
    sub = oracle.hausdorff(A[ia], B[ib])
    assert rel(r["H"], sub["H"]) <= 1e-5, (i, r["H"], sub["H"])
    d = np.sqrt(((A[r["wit_a"]].astype(np.float64) - B[r["wit_b"]]) ** 2).sum())
    assert d == pytest.approx(r["H"], rel=1e-12)
    if not check_dirs:
        return
    o, oe, _ = oracle.directions(A, B, m=m, seed=0)
    # centroid axis: FP32 pilot-shifted sums (same bound as the single-pair test)
    s = A[:4096].astype(np.float64).mean(0)
    mA = np.abs(A.astype(np.float64) - s).mean(0)
    mB = np.abs(B.astype(np.float64) - s).mean(0)
    delta = B.astype(np.float64).mean(0) - A.astype(np.float64).mean(0)
    if np.linalg.norm(delta) > 1e-6:
        bound = 2 * np.linalg.norm(64 * 2.0**-24 * (mA + mB)) / np.linalg.norm(delta) + 1e-12
        assert np.linalg.norm(dirs[0] - o[0]) <= bound
    U = dirs[1:]
    np.testing.assert_allclose(U @ U.T, np.eye(m), atol=1e-12)
    _, C = oracle.union_covariance(A, B)
    w, V = np.linalg.eigh(C)
    lam, V = w[::-1], V[:, ::-1]
    ritz = np.einsum("ld,de,le->l", U, C, U)
    np.testing.assert_allclose(ritz, lam[:m], rtol=0, atol=1.5e-5 * lam[0])
    np.testing.assert_allclose(ritz, oe, rtol=0, atol=1.5e-5 * lam[0])
    for l in range(1, m + 1):
        # against the exact eigenvector (the oracle's deflated power iteration
        # can stop at its iteration cap when lambda_{l+1}/lambda_l is near 1)
        below = lam[l - 1] - lam[l] if l < lam.size else np.inf
        gap = min(below, lam[l - 2] - lam[l - 1] if l >= 2 else np.inf)
        tolang = (1e-5 + 2e-6) * lam[0] / gap
        if tolang < 0.05:
            assert _angle(U[l - 1], V[:, l - 1]) <= tolang, (i, l, _angle(U[l - 1], V[:, l - 1]), tolang)
        # sign convention: the largest |entry| (lowest index on ties) is positive
        j = int(np.argmax(np.abs(U[l - 1])))
        assert U[l - 1, j] > 0

@pytest.mark.parametrize("precision", ["fp16", "bf16", "fp32"])
def test_batch_matches_oracle_per_pair(precision):
    # fp16 / bf16: tensor-core subset HD with margins and FP32 rescoring;
    # fp32: direct differences; the same H within FP32 rounding either way
    pairs = _pairs(SPEC)
    b, res = _run(pairs, precision=precision)
    for i, ((A, B), r) in enumerate(zip(pairs, res)):
        _check_pair(b, i, A, B, r, 8, 0.01, check_dirs=precision == "fp16" and A.shape[0] * A.shape[1] < 3e6)


def test_batch_graph_replay_is_deterministic():
    # the graph and the direct launches run the same kernels on the same tables
    pairs = _pairs(SPEC[:6], seed=5)
    torch = torch_cuda()
    dpairs = [(dev(A), dev(B)) for A, B in pairs]
    b = prohd.Batch(ctx(), dpairs, m=8, alpha_c=0.01)
    b.use_graph(False)
    b.run()
    torch.cuda.synchronize()
    r0 = b.results()
    b.use_graph(True)
    for _ in range(3):
        b.run()
    torch.cuda.synchronize()
    r1 = b.results()
    assert r0 == r1


@pytest.mark.parametrize("tune", [(4096, 4096, 4096), (32768, 32768, 131072)])
def test_batch_tunables_keep_results_exact(tune):
    pairs = _pairs(SPEC[:5], seed=9)
    b, res = _run(pairs, tune=tune)
    for i, ((A, B), r) in enumerate(zip(pairs, res)):
        _check_pair(b, i, A, B, r, 8, 0.01, check_dirs=False)


def test_batch_autotune_then_run():
    torch = torch_cuda()
    pairs = _pairs(SPEC[:4], seed=3)
    dpairs = [(dev(A), dev(B)) for A, B in pairs]
    b = prohd.Batch(ctx(), dpairs, m=8, alpha_c=0.01)
    ms = b.autotune()
    assert ms > 0
    t = b.tunables()
    assert t["gram_pts"] in (4096, 8192, 16384, 32768)
    b.run()
    torch.cuda.synchronize()
    for i, ((A, B), r) in enumerate(zip(pairs, b.results())):
        _check_pair(b, i, A, B, r, 8, 0.01, check_dirs=False)


def test_tuning_table_round_trip(tmp_path):
    # the autotuner's item sizes written to a table file and read into a new
    # context become the defaults of its plans; a table of another device is
    # refused and leaves the context unchanged
    torch_cuda()
    pairs = _pairs(SPEC[:4], seed=5)
    dpairs = [(dev(A), dev(B)) for A, B in pairs]
    c0 = ctx()
    b = prohd.Batch(c0, dpairs, m=8, alpha_c=0.01)
    b.set_tunables(8192, 32768, 4096)
    b.autotune()
    t = b.tunables()
    path = tmp_path / "tunables.txt"
    c0.tunables_save(str(path))
    text = path.read_text()
    assert text.startswith("prohd-tunables 1\n")
    c1 = prohd.Context()
    c1.tunables_load(str(path))
    assert prohd.Batch(c1, dpairs, m=8, alpha_c=0.01).tunables() == t
    other = path.with_name("other.txt")
    lines = text.splitlines()
    lines[1] = "device Another_GPU sms 1 cc 1.0"
    other.write_text("\n".join(lines) + "\n")
    c2 = prohd.Context()
    before = prohd.Batch(c2, dpairs, m=8, alpha_c=0.01).tunables()
    with pytest.raises(prohd.ProHDError):
        c2.tunables_load(str(other))
    with pytest.raises(prohd.ProHDError):
        c2.tunables_load(str(tmp_path / "missing.txt"))
    assert prohd.Batch(c2, dpairs, m=8, alpha_c=0.01).tunables() == before


def test_batch_nonfinite_pair_is_reported_alone():
    pairs = _pairs(SPEC[:4], seed=11)
    A, B = pairs[2]
    A = A.copy()
    A[A.shape[0] // 2, 3] = np.nan
    pairs[2] = (A, B)
    b, res = _run(pairs)
    assert res[2]["status"] == "ENONFINITE"
    for i in (0, 1, 3):
        _check_pair(b, i, pairs[i][0], pairs[i][1], res[i], 8, 0.01, check_dirs=False)


def test_batch_small_alpha_and_m():
    # k = 1 everywhere (alpha n < 1) and m = 2
    pairs = _pairs([(500, 700, 64), (90, 80, 128), (3000, 10, 256)], seed=21)
    b, res = _run(pairs, m=2, alpha=0.0005)
    for i, ((A, B), r) in enumerate(zip(pairs, res)):
        _check_pair(b, i, A, B, r, 2, 0.0005, check_dirs=False)
    b, res = _run(pairs, m=2, alpha=0.0005, precision="fp32")
    for i, ((A, B), r) in enumerate(zip(pairs, res)):
        _check_pair(b, i, A, B, r, 2, 0.0005, check_dirs=False)


def test_batch_rejects_bad_pairs():
    torch = torch_cuda()
    A = dev(np.zeros((10, 13), np.float32))
    with pytest.raises(prohd.ProHDError, match="ENOTSUP"):
        prohd.Batch(ctx(), [(A, A)], m=2, alpha_c=0.1)
    A = dev(np.zeros((10, 16), np.float32))
    with pytest.raises(prohd.ProHDError, match="ENOTSUP"):
        prohd.Batch(ctx(), [(A, A)], m=30, alpha_c=0.1)
    with pytest.raises(prohd.ProHDError, match="EINVAL"):
        prohd.Batch(ctx(), [(A, A)], m=2, alpha_c=0.1, refine=2)
    torch.cuda.synchronize()


@pytest.mark.parametrize("precision", ["fp16", "bf16", "fp32"])
def test_batch_refined_matches_oracle_per_pair(precision):
    # params.refine = 1 in a batch: per pair max(h(A_sel, B), h(B_sel, A))
    # over the batch's own candidate sets, each within 1e-5 of the oracle's
    # refinement of those sets; the witness is a selected point at distance
    # H1 (FP64); H1 never exceeds the exact H of the pair; the candidate sets
    # are those of the plain batch
    spec = SPEC[:3] + [(1, 5, 64), (300, 20_000, 256), (2000, 3000, 8), (1500, 60_000, 96)]
    pairs = _pairs(spec, seed=13)
    torch = torch_cuda()
    dpairs = [(dev(A), dev(B)) for A, B in pairs]
    b0 = prohd.Batch(ctx(), dpairs, m=8, alpha_c=0.01, precision=precision)
    b0.run()
    b1 = prohd.Batch(ctx(), dpairs, m=8, alpha_c=0.01, precision=precision, refine=1)
    b1.run()
    torch.cuda.synchronize()
    for i, ((A, B), r0, r) in enumerate(zip(pairs, b0.results(), b1.results())):
        assert r["status"] == "OK", (i, r["status"])
        assert (r["nsel_a"], r["nsel_b"]) == (r0["nsel_a"], r0["nsel_b"])
        _, ia, ib = b1.pair_outputs(i, r["nsel_a"], r["nsel_b"])
        _, ia0, ib0 = b0.pair_outputs(i, r0["nsel_a"], r0["nsel_b"])
        np.testing.assert_array_equal(ia, ia0)
        np.testing.assert_array_equal(ib, ib0)
        o = oracle.refined(A, B, ia, ib)
        assert rel(r["h_ab"], o["h_ab"]) <= 1e-5, (i, r["h_ab"], o["h_ab"])
        assert rel(r["h_ba"], o["h_ba"]) <= 1e-5, (i, r["h_ba"], o["h_ba"])
        assert rel(r["H"], o["H1"]) <= 1e-5, (i, r["H"], o["H1"])
        d = np.sqrt(((A[r["wit_a"]].astype(np.float64) - B[r["wit_b"]]) ** 2).sum())
        assert d == pytest.approx(r["H"], rel=1e-12)
        sel = set(ia.tolist()) if r["dir"] == 0 else set(ib.tolist())
        assert (r["wit_a"] if r["dir"] == 0 else r["wit_b"]) in sel
        if A.shape[0] * B.shape[0] <= 2e7:
            assert r["H"] <= oracle.hausdorff(A, B)["H"] * (1 + 1e-6)


def test_batch_refined_graph_replay_is_deterministic():
    pairs = _pairs(SPEC[:4], seed=17)
    torch = torch_cuda()
    dpairs = [(dev(A), dev(B)) for A, B in pairs]
    b = prohd.Batch(ctx(), dpairs, m=8, alpha_c=0.01, refine=1)
    b.use_graph(False)
    b.run()
    torch.cuda.synchronize()
    r0 = b.results()
    b.use_graph(True)
    for _ in range(2):
        b.run()
    torch.cuda.synchronize()
    assert b.results() == r0
