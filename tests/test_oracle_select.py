"""Pins for the oracle's extreme selection (Algorithms 1-2), Algorithm 3, and
the bounds of Methodology – Theoretical Properties."""
import numpy as np
import pytest

import oracle
from paper_2511_18207_gb300 import workloads as W


def _brute_select(X, dirs, ks):
    X64 = X.astype(np.float64)
    chosen = set()
    for u, k in zip(np.atleast_2d(dirs), ks):
        p = [float(sum(float(x[j]) * float(u[j]) for j in range(X.shape[1]))) + 0.0 for x in X64]
        order = sorted(range(len(p)), key=lambda i: (p[i], i))
        chosen.update(order[:k])
        order = sorted(range(len(p)), key=lambda i: (-p[i], i))
        chosen.update(order[:k])
    return np.array(sorted(chosen), dtype=np.int64)


def test_k_rule():
    assert oracle.k_of(0.01, 2000) == 20
    assert oracle.k_of(0.01, 99) == 1   # max(1, floor(0.99))
    assert oracle.k_of(0.5, 1) == 1
    assert oracle.k_of(0.02, 2000) == 40
    assert oracle.k_of(0.01 / 8, 2_000_000) == 2500


@pytest.mark.parametrize("seed", range(15))
def test_select_against_brute_force(seed):
    rng = np.random.default_rng(seed)
    n, D = int(rng.integers(1, 40)), int(rng.integers(1, 5))
    # integer-valued points force exact ties
    X = rng.integers(-3, 4, (n, D)).astype(np.float32)
    dirs = rng.standard_normal((3, D))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    ks = [int(rng.integers(1, n + 1)) for _ in range(3)]
    np.testing.assert_array_equal(oracle.select(X, dirs, ks), _brute_select(X, dirs, ks))


def test_select_properties():
    rng = np.random.default_rng(7)
    X = rng.standard_normal((50, 3)).astype(np.float32)
    u = np.array([[0.6, 0.8, 0.0]])
    # sign invariance: -u swaps bottom and top, union unchanged
    np.testing.assert_array_equal(oracle.select(X, u, [5]), oracle.select(X, -u, [5]))
    # distinct projections: exactly 2k points
    assert oracle.select(X, u, [5]).size == 10
    # k >= n/2 keeps everything
    assert oracle.select(X, u, [25]).size == 50
    # duplicates: all points equal, ties by lowest index at both ends
    Y = np.zeros((10, 2), dtype=np.float32)
    np.testing.assert_array_equal(oracle.select(Y, np.array([[1.0, 0.0]]), [3]), [0, 1, 2])


def test_alg3_subset_examples(golden):
    g = golden("alg3_subset_examples.json")
    for c in g["cases"]:
        A = np.asarray(c["A"], dtype=np.float32)
        B = np.asarray(c["B"], dtype=np.float32)
        dirs = np.asarray(c["dirs"], dtype=np.float64)
        ia = oracle.select(A, dirs, c["k"])
        ib = oracle.select(B, dirs, c["k"])
        np.testing.assert_array_equal(ia, c["idxA"], err_msg=c["name"])
        np.testing.assert_array_equal(ib, c["idxB"], err_msg=c["name"])
        assert oracle.hausdorff(A, B)["H"] == pytest.approx(c["H"], abs=1e-12)
        assert oracle.hausdorff(A[ia], B[ib])["H"] == pytest.approx(c["H_hat"], abs=1e-12)
        if "H_u" in c:
            assert oracle.H_u(A, B, dirs[0]) == pytest.approx(c["H_u"], abs=1e-12)


@pytest.mark.slow
def test_table2_random_clouds_count(golden):
    g = golden("table2_random_clouds.json")
    for seed in g["seeds"]:
        A, B = W.random_clouds(g["n_a"], g["n_b"], g["D"], g["offset"], seed=seed)
        r = oracle.prohd(A, B, alpha=g["alpha"], m=g["m"], seed=0)
        assert r["idxA"].size + r["idxB"].size == g["total_selected"], seed


def test_hhat_equals_h_when_everything_is_kept():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((9, 3)).astype(np.float32)
    B = (rng.standard_normal((7, 3)) + 1).astype(np.float32)
    r = oracle.prohd(A, B, alpha=0.6, m=1)  # 2k >= n on every direction
    assert r["idxA"].size == 9 and r["idxB"].size == 7
    assert r["H_hat"] == oracle.hausdorff(A, B)["H"]


@pytest.mark.parametrize("seed", range(8))
def test_sec3e_bounds(seed):
    # H_u <= H <= H_U + 2 min_u delta(u), and monotonicity of H_U in U
    rng = np.random.default_rng(200 + seed)
    A = rng.standard_normal((30, 3)).astype(np.float32)
    B = (rng.standard_normal((25, 3)) * 1.5 + 0.4).astype(np.float32)
    dirs, _, _ = oracle.directions(A, B, m=2)
    H = oracle.hausdorff(A, B)["H"]
    Hu = [oracle.H_u(A, B, u) for u in dirs]
    dl = [oracle.delta(A, B, u) for u in dirs]
    for h in Hu:
        assert h <= H + 1e-12
    assert H <= max(Hu) + 2 * min(dl) + 1e-12
    assert max(Hu[:1]) <= max(Hu[:2]) <= max(Hu) <= H + 1e-12


def test_overestimate_is_possible_and_reported():
    # Methodology – Intuition and Theoretical Properties state H_hat <= H; with subset-vs-subset HD (Algorithm 3)
    # it can exceed H. Count such cases on tiny random inputs: they exist.
    rng = np.random.default_rng(0)
    over = 0
    for _ in range(300):
        A = rng.standard_normal((8, 2)).astype(np.float32)
        B = rng.standard_normal((8, 2)).astype(np.float32)
        r = oracle.prohd(A, B, alpha=0.13, m=1)
        if r["H_hat"] > oracle.hausdorff(A, B)["H"] + 1e-9:
            over += 1
    assert over > 0


def test_delta_closed_form():
    # Eq. 2: distance of the farthest point from the line spanned by u
    A = np.array([[1.0, 0.0], [5.0, 0.0]], dtype=np.float32)
    B = np.array([[2.0, 3.0], [-1.0, -2.0]], dtype=np.float32)
    assert oracle.delta(A, A, np.array([1.0, 0.0])) == 0.0
    assert oracle.delta(A, B, np.array([1.0, 0.0])) == 3.0
    assert oracle.delta(A, B, np.array([0.0, 1.0])) == 5.0


def _brute_one_sided(X, Y, idx):
    best, wi, wj = -1.0, -1, -1
    for i in idx:
        dmin, jmin = None, -1
        for j in range(Y.shape[0]):
            d = float(np.sqrt(sum((float(X[i, c]) - float(Y[j, c])) ** 2 for c in range(X.shape[1]))))
            if dmin is None or d < dmin:
                dmin, jmin = d, j
        if dmin > best:
            best, wi, wj = dmin, int(i), jmin
    return best, wi, wj


@pytest.mark.parametrize("seed", range(4))
def test_refined_against_brute_force(seed):
    rng = np.random.default_rng(40 + seed)
    A = rng.standard_normal((13, 3)).astype(np.float32)
    B = (rng.standard_normal((11, 3)) + 0.7).astype(np.float32)
    ia = np.array(sorted(rng.choice(13, 5, replace=False)))
    ib = np.array(sorted(rng.choice(11, 4, replace=False)))
    r = oracle.refined(A, B, ia, ib)
    h_ab, a1, b1 = _brute_one_sided(A, B, ia)
    h_ba, b2, a2 = _brute_one_sided(B, A, ib)
    assert r["h_ab"] == pytest.approx(h_ab, rel=1e-12)
    assert r["h_ba"] == pytest.approx(h_ba, rel=1e-12)
    assert r["H1"] == max(r["h_ab"], r["h_ba"])
    # the witness is a pair of the original sets at distance H1
    wa, wb = (a1, b1) if h_ab >= h_ba else (a2, b2)
    assert (r["wit_a"], r["wit_b"]) == (wa, wb)


def test_refined_one_dimensional_closed_form():
    # A = {0, 5, 10}, B = {0, 10}: H = 5 (the middle point of A); the
    # extremes alone see no gap, the middle point brings H back
    A = np.array([[0.0], [5.0], [10.0]], dtype=np.float32)
    B = np.array([[0.0], [10.0]], dtype=np.float32)
    assert oracle.hausdorff(A, B)["H"] == 5.0
    assert oracle.refined(A, B, [0, 2], [0, 1])["H1"] == 0.0
    r = oracle.refined(A, B, [1], [0])
    assert r["H1"] == 5.0 and r["wit_a"] == 1 and r["dir"] == 0


def test_refined_never_exceeds_h_and_grows_with_the_subsets():
    # on the tiny trials where Algorithm 3's subset HD overshoots H, the
    # one-sided form stays below H; enlarging either subset cannot lower it;
    # keeping every point gives H exactly
    rng = np.random.default_rng(0)
    over = 0
    for _ in range(300):
        A = rng.standard_normal((8, 2)).astype(np.float32)
        B = rng.standard_normal((8, 2)).astype(np.float32)
        H = oracle.hausdorff(A, B)["H"]
        p = oracle.prohd(A, B, alpha=0.13, m=1)
        over += p["H_hat"] > H + 1e-9
        r = oracle.refined(A, B, p["idxA"], p["idxB"])
        assert r["H1"] <= H + 1e-12
        big = oracle.refined(A, B, np.union1d(p["idxA"], [3]), p["idxB"])
        assert big["H1"] >= r["H1"]
    assert over > 0
    A = rng.standard_normal((9, 4)).astype(np.float32)
    B = rng.standard_normal((6, 4)).astype(np.float32)
    assert oracle.refined(A, B, np.arange(9), np.arange(6))["H1"] == oracle.hausdorff(A, B)["H"]


def test_adaptive_alpha_hand_derived(golden):
    g = golden("adaptive_alpha_1d.json")
    A = np.array(g["A"], dtype=np.float32)
    B = np.array(g["B"], dtype=np.float32)
    assert oracle.hausdorff(A, B)["H"] == 4.0
    for c in g["cases"]:
        r = oracle.adaptive(A, B, g["alpha"], c["alpha_max"], c["rel_tol"], dirs=g["dirs"])
        assert r["H"] == c["H"], c
        assert r["nsel_a"] == c["nsel_a"] and all(n == 2 for n in r["nsel_b"])
        assert r["reason"] == c["reason"] and r["steps"] == len(c["H"])
        assert r["alpha"] == pytest.approx(c["alpha"], rel=1e-15)


def _brute_adaptive(A, B, dirs, alpha, alpha_max, rel_tol):
    # selection by full sorts, refined estimate by nested loops
    Hs = []
    t = 0
    while True:
        a_t = alpha * 2.0**t
        ks = [max(1, min(int(np.floor(a_t * A.shape[0])), A.shape[0]))] * len(dirs)
        kb = [max(1, min(int(np.floor(a_t * B.shape[0])), B.shape[0]))] * len(dirs)
        ia, ib = _brute_select(A, dirs, ks), _brute_select(B, dirs, kb)
        h = max(_brute_one_sided(A, B, ia)[0], _brute_one_sided(B, A, ib)[0])
        Hs.append(h)
        if ia.size == A.shape[0] and ib.size == B.shape[0]:
            return Hs, "all"
        if t >= 1 and Hs[-1] - Hs[-2] <= rel_tol * Hs[-1]:
            return Hs, "stable"
        if alpha * 2.0 ** (t + 1) > alpha_max:
            return Hs, "budget"
        t += 1


@pytest.mark.parametrize("seed", range(4))
def test_adaptive_alpha_against_brute_force(seed):
    rng = np.random.default_rng(70 + seed)
    A = rng.standard_normal((23, 3)).astype(np.float32)
    B = (rng.standard_normal((17, 3)) * 1.3 + 0.5).astype(np.float32)
    dirs = rng.standard_normal((2, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    for alpha_max, tol in [(0.99, 0.0), (0.3, 0.0), (0.99, 0.05)]:
        # alpha_p = alpha on the second direction, as the brute force takes it
        r = oracle.adaptive(A, B, 0.05, alpha_max, tol, dirs=dirs, alpha_p=0.05)
        Hs, why = _brute_adaptive(A, B, dirs, 0.05, alpha_max, tol)
        assert r["reason"] == why and r["steps"] == len(Hs)
        np.testing.assert_allclose(r["H"], Hs, rtol=1e-12)


def test_adaptive_alpha_invariants():
    # non-decreasing, never above H, and equal to H once every point is kept
    A, B = W.random_clouds(300, 200, 3, seed=4)
    H = oracle.hausdorff(A, B)["H"]
    r = oracle.adaptive(A, B, 0.005, 0.99, 0.0, m=1)
    assert all(b >= a for a, b in zip(r["H"], r["H"][1:]))
    assert max(r["H"]) <= H + 1e-12
    assert r["reason"] in ("all", "stable")
    if r["reason"] == "all":
        assert r["H1"] == H
    assert all(b >= a for a, b in zip(r["nsel_a"], r["nsel_a"][1:]))
