"""Pins for the oracle's exact Hausdorff distance (Eq. 1).

The oracle is checked against hand-derived values, scipy's independent
implementation, brute force written differently (numpy broadcasting), and the
metric properties of H on finite sets."""
import numpy as np
import pytest

import oracle


def test_closed_forms(golden):
    g = golden("hd_closed_forms.json")
    for c in g["cases"]:
        A = np.asarray(c["A"], dtype=np.float32)
        B = np.asarray(c["B"], dtype=np.float32)
        h_ab = oracle.directed_hd(A, B)[0]
        h_ba = oracle.directed_hd(B, A)[0]
        if "h_ab" in c:
            assert h_ab == pytest.approx(c["h_ab"], abs=1e-12), c["name"]
        if "h_ba" in c:
            assert h_ba == pytest.approx(c["h_ba"], abs=1e-12), c["name"]
        if "h_ba_sq" in c:
            assert h_ba * h_ba == pytest.approx(c["h_ba_sq"], rel=1e-12), c["name"]


@pytest.mark.parametrize("seed", range(20))
def test_against_scipy_and_numpy(seed):
    from scipy.spatial.distance import directed_hausdorff

    rng = np.random.default_rng(seed)
    D = int(rng.integers(1, 6))
    A = rng.standard_normal((int(rng.integers(1, 12)), D)).astype(np.float32)
    B = (rng.standard_normal((int(rng.integers(1, 12)), D)) + 0.3).astype(np.float32)
    h, i, j = oracle.directed_hd(A, B)
    ref = directed_hausdorff(A.astype(np.float64), B.astype(np.float64))[0]
    assert h == pytest.approx(ref, rel=1e-12, abs=1e-12)
    d = np.sqrt(((A[:, None, :].astype(np.float64) - B[None, :, :]) ** 2).sum(-1))
    assert h == pytest.approx(d.min(1).max(), rel=1e-12, abs=1e-12)
    # witness: i attains the max of row minima, j is i's nearest neighbour
    assert d[i, j] == pytest.approx(h, rel=1e-12, abs=1e-12)
    assert i == int(np.argmax(d.min(1)))


def test_rows_and_witness_tiebreak():
    # two rows tie for the max and two columns tie for the min: lowest indices win
    A = np.array([[0.0], [2.0], [-2.0]], dtype=np.float32)
    B = np.array([[1.0], [-1.0]], dtype=np.float32)
    h, i, j, rm, ra = oracle.directed_hd(A, B, want_rows=True)
    assert h == 1.0 and i == 0 and j == 0
    assert list(rm) == [1.0, 1.0, 1.0] and list(ra) == [0, 0, 1]


def test_row_range_matches_full():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((40, 7)).astype(np.float32)
    B = rng.standard_normal((30, 7)).astype(np.float32)
    _, _, _, rm, _ = oracle.directed_hd(A, B, want_rows=True)
    h2, i2, _ = oracle.directed_hd(A, B, row_begin=10, row_end=25)
    assert h2 == pytest.approx(np.sqrt(rm[10:25].max()), rel=1e-15)
    assert 10 <= i2 < 25


@pytest.mark.parametrize("seed", range(10))
def test_metric_invariants(seed):
    rng = np.random.default_rng(100 + seed)
    D = 4
    A = rng.standard_normal((15, D)).astype(np.float32)
    B = (rng.standard_normal((11, D)) * 2.0).astype(np.float32)
    C = (rng.standard_normal((9, D)) + 1.0).astype(np.float32)
    H = lambda X, Y: oracle.hausdorff(X, Y)["H"]
    # symmetry, identity
    assert H(A, B) == H(B, A)
    assert H(A, A) == 0.0
    # triangle inequality (HD is a metric on finite sets)
    assert H(A, C) <= H(A, B) + H(B, C) + 1e-12
    # translation by an exactly representable vector
    t = np.array([0.5, -1.0, 2.0, 0.25], dtype=np.float32)
    assert H(A + t, B + t) == pytest.approx(H(A, B), rel=1e-6)
    # rotation (float32 rounding of the rotated points bounds the difference)
    Q, _ = np.linalg.qr(rng.standard_normal((D, D)))
    Ar = (A.astype(np.float64) @ Q).astype(np.float32)
    Br = (B.astype(np.float64) @ Q).astype(np.float32)
    assert H(Ar, Br) == pytest.approx(H(A, B), rel=1e-5)


def test_one_dimensional_closed_form():
    # for 1D sets, h(A,B) equals the brute-force 1D HD of the projections on e_1
    rng = np.random.default_rng(5)
    A = rng.uniform(0, 10, (25, 1)).astype(np.float32)
    B = rng.uniform(0, 10, (17, 1)).astype(np.float32)
    u = np.array([1.0])
    assert oracle.directed_hd(A, B)[0] == pytest.approx(
        oracle.hd_1d(oracle.project(A, u), oracle.project(B, u)), rel=1e-15)
    # and for sorted B, the NN of a is a neighbour in sort order
    b = np.sort(B[:, 0].astype(np.float64))
    best = 0.0
    for a in A[:, 0].astype(np.float64):
        k = np.searchsorted(b, a)
        cands = [abs(a - b[k2]) for k2 in (k - 1, k) if 0 <= k2 < b.size]
        best = max(best, min(cands))
    assert oracle.directed_hd(A, B)[0] == pytest.approx(best, rel=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_row_pruning_scheme_keeps_the_row_attaining_h(seed):
    # The scheme of the pruned exact distance, in FP64 on small sets: sampled
    # rows give lower bounds of h(X, Y); every row's NN distance over a
    # prefix of Y bounds its NN distance from above; the rows whose bound
    # reaches the largest lower bound keep h(X, Y) exactly.
    rng = np.random.default_rng(90 + seed)
    X = (rng.standard_normal((3000, 6)) * np.linspace(2, 0.3, 6)).astype(np.float32)
    Y = (rng.standard_normal((2500, 6)) * np.linspace(2, 0.3, 6) + 0.2).astype(np.float32)
    h, _, _, nn, _ = oracle.directed_hd(X, Y, want_rows=True)
    nn = np.sqrt(nn)
    sample1 = (np.arange(64) * X.shape[0]) // 64
    lb1 = nn[sample1].max()
    prefix = np.sqrt(((X[:, None, :].astype(np.float64) - Y[None, :256, :]) ** 2).sum(-1)).min(1)
    assert np.all(prefix >= nn - 1e-12)
    hard = np.flatnonzero(prefix >= lb1)
    lb2 = nn[hard[(np.arange(min(64, hard.size)) * hard.size) // min(64, hard.size)]].max()
    kept = np.flatnonzero(prefix >= max(lb1, lb2) * (1 - 1e-4))
    assert kept.size < X.shape[0]
    assert nn[kept].max() == h
    assert oracle.directed_hd(X[kept], Y)[0] == h
