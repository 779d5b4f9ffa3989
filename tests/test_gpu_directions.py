"""GPU directions (Algorithms 1-2) against the FP64 oracle.

Centroid axis: the GPU sums FP32-centred values z - s in FP32 partials of at
most 16 terms before FP64, so each component of a set's mean is within
16 * 2^-24 * mean|z - s| of the FP64 mean; the axis error is then at most
2 ||err(ybar - xbar)|| / ||ybar - xbar||, the bound asserted below.
Principal components are compared by angle. The oracle's power iteration
stops when 1 - |cos| between steps falls below tol, leaving about
sqrt(2 tol)/(1 - ratio) (ratio = lambda_{l+1}/lambda_l). The GPU's block
iteration stops when every returned Ritz pair has residual
||C x - theta x|| <= 2e-6 lambda_1, which bounds its angle to the exact
eigenvector by 2e-6 lambda_1 / gap_l. The GPU's covariance is accumulated on
tensor cores from an exact three-way BF16 split of every centred value (six
products, each within ~2^-24 of z_i z_j), summed in FP32 over 512 points
(3072 exact products; random-walk error ~sqrt(3072) 2^-24 = 3.3e-6 relative)
and in FP64 beyond; 1e-5 ||C|| (3x that) bounds the perturbation, which moves
component l by at most that over its eigengap and eigenvalue l by at most that
absolutely."""
import numpy as np
import pytest

import oracle
from paper_2511_18207_gb300 import workloads as W

from .gpu_util import ctx, dev, torch_cuda

pytestmark = pytest.mark.gpu


def _angle(u, v):
    c = abs(float(np.dot(u, v)) / (np.linalg.norm(u) * np.linalg.norm(v)))
    return float(np.arccos(min(c, 1.0)))


def _axis_bound(A, B):
    s = A[:4096].astype(np.float64).mean(0).astype(np.float32).astype(np.float64)
    mA = np.abs(A.astype(np.float64) - s).mean(0)
    mB = np.abs(B.astype(np.float64) - s).mean(0)
    delta = B.astype(np.float64).mean(0) - A.astype(np.float64).mean(0)
    err = 16 * 2.0**-24 * (mA + mB)
    return 2 * np.linalg.norm(err) / np.linalg.norm(delta)


def _gpu_dirs(A, B, m, seed=0):
    torch = torch_cuda()
    d, e = ctx().prohd_directions(dev(A), dev(B), m=m, seed=seed)
    torch.cuda.synchronize()
    return d.cpu().numpy(), e.cpu().numpy()


@pytest.mark.parametrize(
    "D,m,nA,nB",
    [(8, 2, 6000, 5000), (32, 4, 6000, 5000), (64, 8, 6000, 5000), (256, 8, 6000, 5000), (100, 5, 6000, 5000),
     (13, 3, 6000, 5000), (300, 4, 6000, 5000), (124, 3, 6000, 5000), (160, 4, 6000, 5000), (192, 6, 6000, 5000),
     # many 64-point chunks per CTA, ragged tails, both CTA types
     (256, 4, 120_000, 90_001), (192, 3, 70_001, 99_999)],
)
def test_directions_anisotropic(D, m, nA, nB):
    # anisotropic Gaussian with eigenvalues 1/i: well separated top components
    A, B = W.anisotropic_pair(nA, nB, D, seed=D)
    g, ge = _gpu_dirs(A, B, m)
    o, oe, _ = oracle.directions(A, B, m=m, seed=0)
    assert np.linalg.norm(g[0] - o[0]) <= _axis_bound(A, B)
    # full spectrum for the eigengaps
    _, C = oracle.union_covariance(A, B)
    lam = np.sort(np.linalg.eigvalsh(C))[::-1]
    for l in range(1, m + 1):
        ratio = lam[l] / lam[l - 1]
        gap = min(lam[l - 1] - lam[l], lam[l - 2] - lam[l - 1] if l >= 2 else np.inf)
        tolang = 2 * np.sqrt(2e-13) / (1 - ratio) + (1e-5 + 2e-6) * lam[0] / gap + 1e-6 / (1 - ratio)
        assert _angle(g[l], o[l]) <= tolang, (l, _angle(g[l], o[l]), tolang)
        # same sign convention
        assert float(np.dot(g[l], o[l])) > 0
    np.testing.assert_allclose(ge, oe, rtol=0, atol=1e-5 * oe[0])


def test_directions_centroid_fallback_and_small():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((500, 6)).astype(np.float32)
    g, _ = _gpu_dirs(A, A, 2)
    np.testing.assert_array_equal(g[0], np.eye(6)[0])
    # unit norms, orthogonality
    np.testing.assert_allclose(np.linalg.norm(g, axis=1), 1.0, rtol=1e-12)
    assert abs(float(g[1] @ g[2])) < 1e-12


def test_directions_config_small():
    A, B = W.gaussian_outliers(2000, 2000, 16, seed=0)
    g, ge = _gpu_dirs(A, B, 2)
    o, oe, _ = oracle.directions(A, B, m=2, seed=0)
    assert np.linalg.norm(g[0] - o[0]) <= _axis_bound(A, B)
    np.testing.assert_allclose(ge, oe, rtol=0, atol=1e-5 * oe[0])
