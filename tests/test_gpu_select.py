"""GPU extreme selection (Algorithms 1-2) against the oracle's full FP64 sort.

Given the same directions, the selected index sets must be identical (integer
results: bit-exact), including exact ties (lowest index first at both ends),
duplicated points, k >= n/2, and dimensions that are not multiples of 4."""
import numpy as np
import pytest

import oracle
from paper_2511_18207_gb300 import workloads as W

from .gpu_util import ctx, dev, torch_cuda

pytestmark = pytest.mark.gpu


def _gpu_select(A, B, dirs, kA, kB):
    torch = torch_cuda()
    c = ctx()
    ia, na, ib, nb = c.prohd_select(dev(A), dev(B), torch.from_numpy(np.asarray(dirs, dtype=np.float64)), kA, kB)
    torch.cuda.synchronize()
    na, nb = int(na.item()), int(nb.item())
    return ia[:na].cpu().numpy().astype(np.int64), ib[:nb].cpu().numpy().astype(np.int64)


def _check(A, B, dirs, kA, kB):
    ga, gb = _gpu_select(A, B, dirs, kA, kB)
    np.testing.assert_array_equal(ga, oracle.select(A, dirs, kA))
    np.testing.assert_array_equal(gb, oracle.select(B, dirs, kB))


def _unit(rng, nd, D):
    u = rng.standard_normal((nd, D))
    return u / np.linalg.norm(u, axis=1, keepdims=True)


@pytest.mark.parametrize("nA,nB,D,nd", [(1, 1, 4, 1), (5, 3, 4, 2), (2000, 2000, 16, 3), (1000, 3001, 64, 9),
                                        (777, 1025, 13, 5), (4096, 300, 256, 9), (50_000, 40_000, 32, 4)])
def test_select_random_dirs(nA, nB, D, nd):
    rng = np.random.default_rng(nA + nB + D)
    A = rng.standard_normal((nA, D)).astype(np.float32)
    B = (rng.standard_normal((nB, D)) + 0.1).astype(np.float32)
    dirs = _unit(rng, nd, D)
    kA = [oracle.k_of(0.02, nA)] * nd
    kB = [oracle.k_of(0.03, nB)] * nd
    _check(A, B, dirs, kA, kB)


def test_select_ties_integer_grid():
    # integer coordinates along axis directions: massive exact ties
    rng = np.random.default_rng(1)
    A = rng.integers(-3, 4, (3000, 8)).astype(np.float32)
    B = rng.integers(-2, 3, (2500, 8)).astype(np.float32)
    dirs = np.eye(8)[:4]
    _check(A, B, dirs, [100, 7, 1, 500], [33, 2, 250, 1])


def test_select_all_identical_large_band():
    # every projection equal: the band holds all points (radix path beyond
    # shared memory), and ties go to the lowest indices at both ends
    A = np.ones((5000, 4), dtype=np.float32)
    B = np.ones((3000, 4), dtype=np.float32) * 2
    dirs = np.array([[0.5, 0.5, 0.5, 0.5]])
    _check(A, B, dirs, [40], [1000])


def test_select_k_covers_everything():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((100, 4)).astype(np.float32)
    B = rng.standard_normal((90, 4)).astype(np.float32)
    dirs = _unit(rng, 2, 4)
    ga, gb = _gpu_select(A, B, dirs, [60, 60], [45, 200])
    assert ga.size == 100 and gb.size == 90


def test_select_sign_invariance():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((3000, 20)).astype(np.float32)
    B = rng.standard_normal((2000, 20)).astype(np.float32)
    dirs = _unit(rng, 3, 20)
    a1, b1 = _gpu_select(A, B, dirs, [30] * 3, [20] * 3)
    a2, b2 = _gpu_select(A, B, -dirs, [30] * 3, [20] * 3)
    np.testing.assert_array_equal(a1, a2)
    np.testing.assert_array_equal(b1, b2)


def test_select_table2_count():
    # Table 2 random clouds: 6,000 selected points in total (given the oracle's directions)
    A, B = W.random_clouds(100_000, 100_000, 4, 0.1, seed=0)
    dirs, _, _ = oracle.directions(A, B, m=2, seed=0)
    k = oracle.k_list(100_000, 3, 0.01, 0.005)
    ga, gb = _gpu_select(A, B, dirs, k, k)
    assert ga.size + gb.size == 6000
    np.testing.assert_array_equal(ga, oracle.select(A, dirs, k))
