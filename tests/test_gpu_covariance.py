"""Union covariance (Algorithm 2 step 2) on the GPU against the FP64 oracle.

Error model of the tensor-core path (D <= 256, D % 4 == 0). With z = x - s
(s the FP32 pilot shift, the mean of the first 4096 rows of A), the GPU forms
G = sum_z z z^T and C = G/N - dd^T, d = mean - s. Each z is split into
BF16 parts z = h + m + r (|m| <= 2^-8 |z|, |r| <= 2^-16 |z|) and the tensor
cores give sum (h h^T + h m^T + m h^T):
  - the missing terms m_i m_j + h_i r_j + r_i h_j are rounding residuals with
    zero mean; off the diagonal they cancel over the points (a random walk of
    at most 3 2^-16 |z_i z_j| per point, about 1e-7 of |G_ij| here), and on the
    diagonal their sum z_i^2 - h_i^2 - 2 h_i m_i is added back per point;
  - accumulation: 512 points are summed in FP32 by 64 MMAs, each adding to the
    accumulator with at most one FP32 ulp (2^-23) of error, so a partial is
    within 64 * 2^-23 = 7.6e-6 of sum |z_i z_j| <= sqrt(G_ii G_jj); partials are
    summed in FP32 per CTA and in FP64 across CTAs.
So |C_ij - C*_ij| <= 1e-5 sqrt(G_ii G_jj) / N, with G_ii / N = C*_ii + d_i^2.
The CUDA-core path (other D) multiplies in FP32 and accumulates in FP64, well
inside the same bound."""
import numpy as np
import pytest

import oracle
from paper_2511_18207_gb300 import workloads as W

from .gpu_util import ctx, dev, torch_cuda

pytestmark = pytest.mark.gpu


def _check(A, B, tol=1e-5):
    torch = torch_cuda()
    C, mean = ctx().prohd_covariance(dev(A), dev(B))
    torch.cuda.synchronize()
    C, mean = C.cpu().numpy(), mean.cpu().numpy()
    mu, Co = oracle.union_covariance(A, B)
    s = A[:4096].astype(np.float64).mean(0).astype(np.float32).astype(np.float64)
    d = mu - s
    g = np.diag(Co) + d * d  # G_ii / N
    bound = tol * np.sqrt(np.outer(g, g))
    err = np.abs(C - Co)
    worst = float((err / bound).max())
    assert worst <= 1.0, (worst, np.unravel_index(np.argmax(err / bound), err.shape))
    # the symmetric matrix the eigenvector iteration uses
    np.testing.assert_array_equal(C, C.T)
    # the mean: s plus the FP32-compensated sums in FP64
    assert np.abs(mean - mu).max() <= 1e-6 * (np.abs(mu).max() + np.sqrt(g.max()))
    return worst


@pytest.mark.parametrize(
    "D,nA,nB",
    [(8, 6000, 5000), (64, 30_001, 20_003), (100, 7000, 9001), (128, 40_000, 33_333),  # CTAs split points
     (132, 9000, 8000), (192, 70_001, 99_999), (256, 120_000, 90_001),                  # CTAs split dimensions
     (13, 5000, 4000), (300, 6000, 5000)])                                             # CUDA-core path
def test_covariance_anisotropic(D, nA, nB):
    A, B = W.anisotropic_pair(nA, nB, D, seed=D + 1)
    _check(A, B)


def test_covariance_offset_and_heavy_tails():
    # mean far from zero (the pilot shift carries it) and Student-t tails
    A, B = W.anisotropic_pair(50_000, 40_000, 256, shift_sigma=0.1, t_frac=0.01, nu=3.0, seed=7)
    _check(A + np.float32(30.0), B + np.float32(30.0))


def test_covariance_uneven_sets_and_tiny_set():
    # one set far larger than the other, and a set smaller than one tile
    A, B = W.mixture_pair(100_000, 256, 16, seed=4)
    _check(A, B[:3000])
    _check(A[:37], B[:5])
    A, B = W.mixture_pair(100_000, 64, 8, seed=5)
    _check(A[:50], B)


def test_covariance_exact_on_small_integers():
    # small integers whose first 4096 rows of A sum to zero: the pilot shift
    # is 0, every centred value is exact in BF16 (no low part), every product
    # and every FP32 partial sum is an exact integer, so only the final FP64
    # steps round
    rng = np.random.default_rng(3)
    R = rng.integers(-8, 9, size=(2048, 192))
    A = np.vstack([R, -R, rng.integers(-8, 9, size=(16_000, 192))]).astype(np.float32)
    B = rng.integers(-8, 9, size=(10_000, 192)).astype(np.float32)
    assert _check(A, B, tol=1e-12) <= 1.0
