"""GPU directions (Algorithms 1-2) against the FP64 oracle.

The centroid axis is compared to relative 1e-9 (FP64 sums of FP32 partials).
Principal components are compared by angle: both sides stop when
1 - |cos| between steps falls below tol, which leaves an angle error of about
sqrt(2 tol)/(1 - ratio) each (ratio = lambda_{l+1}/lambda_l); the GPU's FP32
matrix-vector products and FP32 covariance partials add ~1e-6/(gap)."""
import numpy as np
import pytest

import oracle
from paper_2511_18207_gb300 import workloads as W

from .gpu_util import ctx, dev, torch_cuda

pytestmark = pytest.mark.gpu


def _angle(u, v):
    c = abs(float(np.dot(u, v)) / (np.linalg.norm(u) * np.linalg.norm(v)))
    return float(np.arccos(min(c, 1.0)))


def _gpu_dirs(A, B, m, seed=0):
    torch = torch_cuda()
    d, e = ctx().prohd_directions(dev(A), dev(B), m=m, seed=seed)
    torch.cuda.synchronize()
    return d.cpu().numpy(), e.cpu().numpy()


@pytest.mark.parametrize("D,m", [(8, 2), (32, 4), (64, 8), (256, 8), (100, 5)])
def test_directions_anisotropic(D, m):
    # anisotropic Gaussian with eigenvalues 1/i: well separated top components
    A, B = W.anisotropic_pair(6000, 5000, D, seed=D)
    g, ge = _gpu_dirs(A, B, m)
    o, oe, _ = oracle.directions(A, B, m=m, seed=0)
    assert np.abs(g[0] - o[0]).max() <= 1e-9
    for l in range(1, m + 1):
        ratio = oe[l] / oe[l - 1] if l < m else 0.9
        tolang = 4 * np.sqrt(2e-13) / max(1 - ratio, 1e-3) + 1e-4 / max(1 - ratio, 1e-2)
        assert _angle(g[l], o[l]) <= tolang, (l, _angle(g[l], o[l]), tolang)
        # same sign convention
        assert float(np.dot(g[l], o[l])) > 0
    np.testing.assert_allclose(ge, oe, rtol=1e-6)


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
    assert np.abs(g[0] - o[0]).max() <= 1e-9
    np.testing.assert_allclose(ge, oe, rtol=1e-6)
