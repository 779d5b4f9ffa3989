"""Pins for the oracle's directions: centroid axis (Algorithm 1), union
covariance and power-iteration principal components (Algorithm 2)."""
import ctypes

import numpy as np
import pytest

import oracle


def test_splitmix64_published_vector():
    # Published SplitMix64 outputs for seed 1234567 (Steele/Lea/Flood 2014,
    # reference implementation; also the test vector of common ports).
    lib = oracle._load()
    lib.oracle_splitmix64_raw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.oracle_splitmix64_raw.restype = ctypes.c_uint64
    expect = [6457827717110365317, 3203168211198807973, 9817491932198370423,
              4593380528125082431, 16408922859458223821]
    assert [lib.oracle_splitmix64_raw(1234567, c) for c in range(5)] == expect
    # the unit map sends the top 53 bits to [-1, 1)
    v = oracle.splitmix64_unit(1234567, 0, 0)
    assert v == pytest.approx((expect[0] >> 11) / 2.0**53 * 2 - 1, rel=0, abs=0)
    assert -1.0 <= oracle.splitmix64_unit(7, 3, 11) < 1.0


def test_centroid_and_axis():
    A = np.array([[0, 0, 0], [2, 0, 0]], dtype=np.float32)
    B = np.array([[1, 3, 0], [1, 5, 0]], dtype=np.float32)
    np.testing.assert_array_equal(oracle.centroid(A), [1, 0, 0])
    np.testing.assert_array_equal(oracle.centroid(B), [1, 4, 0])
    np.testing.assert_array_equal(oracle.centroid_axis(oracle.centroid(A), oracle.centroid(B)), [0, 1, 0])
    # fallback to e_1 below 1e-9 (Algorithm 1), literal absolute threshold
    np.testing.assert_array_equal(oracle.centroid_axis(np.zeros(3), np.full(3, 1e-10)), [1, 0, 0])
    u = oracle.centroid_axis(np.zeros(3), np.array([3.0, 4.0, 0.0]))
    np.testing.assert_allclose(u, [0.6, 0.8, 0.0], rtol=1e-15)


def test_covariance_against_numpy_and_line():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((300, 5)).astype(np.float32)
    B = (rng.standard_normal((200, 5)) * 3 + 1).astype(np.float32)
    mu, C = oracle.union_covariance(A, B)
    Z = np.vstack([A, B]).astype(np.float64)
    np.testing.assert_allclose(mu, Z.mean(0), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(C, np.cov(Z, rowvar=False, bias=True), rtol=1e-12, atol=1e-13)
    # points on a line t*v + c: C = var(t) v v^T exactly up to rounding
    t = np.arange(-5, 6, dtype=np.float64)
    v = np.array([1.0, 2.0, 2.0]) / 3.0
    P = (t[:, None] * v[None, :] * 3.0 + np.array([1.0, -2.0, 0.5])).astype(np.float32)
    _, C = oracle.union_covariance(P[:6], P[6:])
    np.testing.assert_allclose(C, np.var(t * 3.0) * np.outer(v, v), atol=1e-12)


def _spd(D, lam, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((D, D)))
    return (Q * lam[None, :]) @ Q.T


@pytest.mark.parametrize("seed", range(5))
def test_power_iteration_against_eigh(seed):
    D, m = 12, 4
    lam = np.array([10.0 * 0.8**i for i in range(D)])  # gap ratio 0.8 <= 0.9
    C = _spd(D, lam, seed)
    U, l, it = oracle.power_iteration(C, m, seed=seed, tol=1e-13, maxit=2000)
    w, V = np.linalg.eigh(C)
    # the stop rule bounds 1-|cos| between steps, i.e. a step angle of
    # sqrt(2 tol); the remaining error is that over (1 - ratio), ratio = 0.8
    bound = 4.0 * np.sqrt(2 * 1e-13) / (1 - 0.8)
    for k in range(m):
        ref = V[:, -1 - k]
        cos = abs(float(U[k] @ ref))
        assert np.arccos(min(cos, 1.0)) < bound, (k, cos)
        assert l[k] == pytest.approx(w[-1 - k], rel=1e-12)
        # sign rule: the largest-magnitude entry is positive
        assert U[k][np.argmax(np.abs(U[k]))] > 0
    np.testing.assert_allclose(U @ U.T, np.eye(m), atol=1e-12)
    assert (it < 2000).all()


def test_power_iteration_axis_aligned_and_line():
    # axis-aligned, distinct variances: PCs are the coordinate axes in order
    lam = np.array([1.0, 9.0, 4.0, 0.25])
    U, l, _ = oracle.power_iteration(np.diag(lam), 3, seed=1)
    for k, axis in enumerate([1, 2, 0]):
        assert abs(U[k][axis]) == pytest.approx(1.0, abs=1e-12)
        assert U[k][axis] > 0
    np.testing.assert_allclose(l, [9.0, 4.0, 1.0], rtol=1e-13)
    # data on a line: PC1 is the line
    v = np.array([2.0, -1.0, 2.0]) / 3.0
    U, l, _ = oracle.power_iteration(np.outer(v, v) * 5.0, 1, seed=2)
    assert abs(float(U[0] @ v)) == pytest.approx(1.0, abs=1e-14)


def test_power_iteration_eigen_residual():
    # every returned pair satisfies C u = lambda u to the stopping tolerance
    C = _spd(20, np.linspace(5.0, 0.1, 20) ** 2, 9)
    U, l, _ = oracle.power_iteration(C, 5, seed=3, tol=1e-14, maxit=5000)
    for k in range(5):
        r = C @ U[k] - l[k] * U[k]
        assert np.linalg.norm(r) < 1e-5 * l[0]


def test_directions_shape_and_defaults():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((100, 16)).astype(np.float32)
    B = (rng.standard_normal((80, 16)) + 0.5).astype(np.float32)
    dirs, lam, it = oracle.directions(A, B)
    assert dirs.shape == (1 + 4, 16)  # m = floor(sqrt(16)) = 4
    np.testing.assert_allclose(np.linalg.norm(dirs, axis=1), 1.0, rtol=1e-14)
    assert (np.diff(lam) <= 1e-12).all()
