"""Seeded synthetic point-set generators (host, numpy).

This module only draws inputs; it holds none of ProHD's arithmetic. Both the
CUDA path and the FP64 oracle are fed from it, so it imports neither.

The paper's datasets (CIFAR-10, MNIST, Higgs) are not available; these
generators stand in for them with the shapes and structures the paper's
experiments use (Evaluation – Datasets and Experimental Setup: uniform random clouds with a 0.1 offset) and the
workload families this library is benchmarked on:

* ``gaussian_outliers``  N(0, I) vs N(0.5*1, I) with 1% of B scaled x3
* ``gaussian_mixture``   K-component Gaussian mixtures (means ~ N(0, 4I),
                         diagonal variances ~ U[0.2, 2], equal weights)
* ``anisotropic_pair``   A ~ N(0, Q diag(1/i) Q^T); B the same law shifted by
                         0.1 sigma_r along a random unit r, plus a fraction of
                         multivariate Student-t (nu = 3) points
* ``random_clouds``      U[0,1]^D vs U[0,1]^D + 0.1 (Evaluation – Datasets and Experimental Setup)
* ``batched_pairs``      uneven pairs, log-uniform sizes, D in {64,128,256}
* ``student_t_mixture``  anisotropic Student-t mixtures (learned-direction data)

All arrays are float32, row-major [n, D].
"""
from __future__ import annotations

import math

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def _normal(rng: np.random.Generator, n: int, D: int, chunk: int = 1 << 18) -> np.ndarray:
    out = np.empty((n, D), dtype=np.float32)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        out[s:e] = rng.standard_normal((e - s, D), dtype=np.float32)
    return out


def gaussian_outliers(n_a: int = 2000, n_b: int = 2000, D: int = 16, shift: float = 0.5,
                      outlier_frac: float = 0.01, outlier_scale: float = 3.0, seed: int = 0):
    """A ~ N(0, I_D); B ~ N(shift*1, I_D) with ``outlier_frac`` of B's rows
    (chosen by a seeded permutation) multiplied by ``outlier_scale`` after the
    shift."""
    rng = _rng(seed)
    A = _normal(rng, n_a, D)
    B = _normal(rng, n_b, D) + np.float32(shift)
    n_out = int(round(outlier_frac * n_b))
    if n_out:
        rows = rng.permutation(n_b)[:n_out]
        B[rows] *= np.float32(outlier_scale)
    return A, B


def gaussian_mixture(n: int, D: int, K: int = 16, seed: int = 0, mean_var: float = 4.0,
                     var_lo: float = 0.2, var_hi: float = 2.0) -> np.ndarray:
    """One set from a K-component Gaussian mixture: means ~ N(0, mean_var I),
    per-component diagonal variances ~ U[var_lo, var_hi], equal weights."""
    rng = _rng(seed)
    means = rng.standard_normal((K, D)) * math.sqrt(mean_var)
    sd = np.sqrt(rng.uniform(var_lo, var_hi, size=(K, D)))
    comp = rng.integers(0, K, size=n)
    X = _normal(rng, n, D)
    X *= sd[comp].astype(np.float32)
    X += means[comp].astype(np.float32)
    return X


def mixture_pair(n: int = 200_000, D: int = 256, K: int = 16, seed: int = 0):
    """A and B as independent K-component mixtures (seeds 2s and 2s+1)."""
    return gaussian_mixture(n, D, K, seed=2 * seed), gaussian_mixture(n, D, K, seed=2 * seed + 1)


def random_orthogonal(D: int, rng: np.random.Generator) -> np.ndarray:
    """Q from the QR factorisation of a Gaussian matrix, signs fixed by R's diagonal."""
    G = rng.standard_normal((D, D))
    Q, R = np.linalg.qr(G)
    Q *= np.sign(np.diag(R))[None, :]
    return Q


def anisotropic_pair(n_a: int = 2_000_000, n_b: int = 2_000_000, D: int = 256,
                     shift_sigma: float = 0.1, t_frac: float = 0.001, nu: float = 3.0,
                     seed: int = 0):
    """A ~ N(0, S) with S = Q diag(1/i) Q^T (i = 1..D); B drawn from the same
    law, shifted by 0.1 * sigma_r * r for a random unit r with
    sigma_r = sqrt(r^T S r); ``t_frac`` of B's rows are replaced by
    multivariate Student-t (nu) points with scale matrix S and the same shift.
    """
    rng = _rng(seed)
    Q = random_orthogonal(D, rng)
    lam = 1.0 / np.arange(1, D + 1, dtype=np.float64)
    M = (np.sqrt(lam)[:, None] * Q.T).astype(np.float32)  # rows: x = z @ M
    r = rng.standard_normal(D)
    r /= np.linalg.norm(r)
    sigma_r = math.sqrt(float(r @ (Q * lam[None, :]) @ Q.T @ r))
    shift = (shift_sigma * sigma_r * r).astype(np.float32)

    def draw(n):
        out = np.empty((n, D), dtype=np.float32)
        chunk = 1 << 18
        for s in range(0, n, chunk):
            e = min(n, s + chunk)
            out[s:e] = rng.standard_normal((e - s, D), dtype=np.float32) @ M
        return out

    A = draw(n_a)
    B = draw(n_b)
    B += shift
    n_t = int(round(t_frac * n_b))
    if n_t:
        rows = rng.permutation(n_b)[:n_t]
        z = rng.standard_normal((n_t, D)) @ M.astype(np.float64)
        w = rng.chisquare(nu, size=n_t) / nu
        B[rows] = (z / np.sqrt(w)[:, None]).astype(np.float32) + shift
    return A, B


def random_clouds(n_a: int = 100_000, n_b: int = 100_000, D: int = 4, offset: float = 0.1,
                  seed: int = 0):
    """U[0,1]^D vs U[0,1]^D + offset (Evaluation – Datasets and Experimental Setup random clouds)."""
    rng = _rng(seed)
    A = rng.random((n_a, D), dtype=np.float32)
    B = rng.random((n_b, D), dtype=np.float32) + np.float32(offset)
    return A, B


def batched_pairs(npairs: int = 512, n_lo: int = 1000, n_hi: int = 100_000,
                  dims=(64, 128, 256), k_lo: int = 4, k_hi: int = 32, seed: int = 0):
    """List of (A, B) pairs: sizes log-uniform on [n_lo, n_hi] per set, D drawn
    from ``dims``, each set a mixture of K ~ U{k_lo..k_hi} components with the
    same component law as ``gaussian_mixture``; pair p uses seed + p."""
    pairs = []
    for p in range(npairs):
        rng = _rng(seed * 1_000_003 + p)
        na = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        nb = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        D = int(rng.choice(np.asarray(dims)))
        K = int(rng.integers(k_lo, k_hi + 1))
        s = int(rng.integers(0, 2**31 - 1))
        pairs.append((gaussian_mixture(na, D, K, seed=2 * s), gaussian_mixture(nb, D, K, seed=2 * s + 1)))
    return pairs


def batched_pairs_device(npairs: int = 512, n_lo: int = 1000, n_hi: int = 100_000, dims=(64, 128, 256),
                         k_lo: int = 4, k_hi: int = 32, seed: int = 0, device: str = "cuda"):
    """The law of ``batched_pairs`` drawn with torch generators on the device
    (the benchmark's 512-pair batch holds about 13 GB; drawing it on the host
    would dominate the run). Sizes, D and K come from a seeded CPU generator,
    the points from a seeded device generator: list of (A, B) float32 CUDA
    tensors."""
    import torch

    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    gd = torch.Generator(device=device)
    gd.manual_seed(int(seed) + 1)
    lo, hi = math.log(n_lo), math.log(n_hi)
    pairs = []
    for _ in range(npairs):
        u = torch.rand(2, generator=g, dtype=torch.float64)
        sizes = [int(round(math.exp(lo + float(x) * (hi - lo)))) for x in u]
        D = int(dims[int(torch.randint(0, len(dims), (1,), generator=g))])
        K = int(torch.randint(k_lo, k_hi + 1, (1,), generator=g))
        sets = []
        for n in sizes:
            means = torch.randn(K, D, generator=gd, device=device) * 2.0
            sd = torch.sqrt(torch.empty(K, D, device=device).uniform_(0.2, 2.0, generator=gd))
            comp = torch.randint(0, K, (n,), generator=gd, device=device)
            X = torch.randn(n, D, generator=gd, device=device) * sd[comp] + means[comp]
            sets.append(X.contiguous())
        pairs.append((sets[0], sets[1]))
    return pairs


def student_t_mixture(n: int, D: int = 128, K: int = 8, nu: float = 3.0, seed: int = 0) -> np.ndarray:
    """K-component mixture of anisotropic multivariate Student-t (nu) laws:
    component c has mean ~ N(0, 4I) and scale Q_c diag(1/i) Q_c^T."""
    rng = _rng(seed)
    lam = 1.0 / np.arange(1, D + 1, dtype=np.float64)
    out = np.empty((n, D), dtype=np.float32)
    comp = rng.integers(0, K, size=n)
    for c in range(K):
        rows = np.flatnonzero(comp == c)
        if rows.size == 0:
            continue
        Q = random_orthogonal(D, rng)
        M = np.sqrt(lam)[:, None] * Q.T
        mean = rng.standard_normal(D) * 2.0
        z = rng.standard_normal((rows.size, D)) @ M
        w = rng.chisquare(nu, size=rows.size) / nu
        out[rows] = (z / np.sqrt(w)[:, None] + mean).astype(np.float32)
    return out


def student_t_mixture_device(n: int, D: int = 128, K: int = 8, nu: float = 3.0, seed: int = 0,
                             device: str = "cuda"):
    """The law of ``student_t_mixture`` drawn with torch on the device
    (component rotations from QR of Gaussian matrices, signs fixed by R's
    diagonal): a float32 CUDA tensor [n, D]."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    lam = 1.0 / torch.arange(1, D + 1, dtype=torch.float64, device=device)
    G = torch.randn(K, D, D, generator=g, device=device, dtype=torch.float64)
    Q, R = torch.linalg.qr(G)
    Q = Q * torch.sign(torch.diagonal(R, dim1=1, dim2=2))[:, None, :]
    M = torch.sqrt(lam)[None, :, None] * Q.transpose(1, 2)          # [K, D, D]: x = z @ M_c
    means = torch.randn(K, D, generator=g, device=device, dtype=torch.float64) * 2.0
    comp = torch.randint(0, K, (n,), generator=g, device=device)
    z = torch.randn(n, D, generator=g, device=device, dtype=torch.float64)
    w = _chi2_torch(n, nu, g, device) / nu
    x = torch.empty(n, D, dtype=torch.float64, device=device)
    for c in range(K):
        rows = torch.nonzero(comp == c, as_tuple=True)[0]
        x[rows] = z[rows] @ M[c]
    x = x / torch.sqrt(w)[:, None] + means[comp]
    return x.to(torch.float32).contiguous()


_ROTATION_POOLS = {}


def rotation_pool(D: int, size: int = 64, seed: int = 4242, device: str = "cuda"):
    """A fixed pool of `size` random orthogonal D x D matrices (QR of seeded
    Gaussian matrices, signs fixed by R's diagonal), FP32 on the device,
    drawn once per (D, device)."""
    import torch

    key = (D, size, seed, str(device))
    if key not in _ROTATION_POOLS:
        g = torch.Generator(device="cpu")
        g.manual_seed(int(seed))
        G = torch.randn(size, D, D, generator=g, dtype=torch.float64)
        Q, R = torch.linalg.qr(G)
        Q = Q * torch.sign(torch.diagonal(R, dim1=1, dim2=2))[:, None, :]
        _ROTATION_POOLS[key] = Q.to(device=device, dtype=torch.float32).contiguous()
    return _ROTATION_POOLS[key]


def student_t_mixture_pool(n: int, D: int = 128, K: int = 8, nu: int = 3, seed: int = 0, device: str = "cuda"):
    """Anisotropic Student-t (integer nu) mixture drawn on the device in FP32,
    without host synchronisation: K equally likely components with means
    ~ N(0, 4I); component c draws z ~ N(0, I), x = z diag(1/sqrt(i)) R_c^T,
    with R_c taken from the fixed rotation pool by a seeded index, divided
    by sqrt(chi2_nu / nu). Component sizes are multinomial (seeded CPU
    generator) and the points come in component blocks: the Hausdorff
    distance and ProHD do not depend on the order of the points."""
    import torch

    gc = torch.Generator(device="cpu")
    gc.manual_seed(int(seed))
    counts = torch.bincount(torch.randint(0, K, (n,), generator=gc), minlength=K).tolist()
    rot = torch.randint(0, rotation_pool(D, device=device).shape[0], (K,), generator=gc).tolist()
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    pool = rotation_pool(D, device=device)
    scale = (1.0 / torch.arange(1, D + 1, dtype=torch.float32, device=device)).sqrt()
    means = torch.randn(K, D, generator=g, device=device) * 2.0
    z = torch.randn(n, D, generator=g, device=device)
    w = (torch.randn(n, nu, generator=g, device=device) ** 2).sum(1) / nu
    x = torch.empty(n, D, dtype=torch.float32, device=device)
    off = 0
    for c in range(K):
        m = counts[c]
        if m:
            M = scale[:, None] * pool[rot[c]].t()  # x = z @ M
            torch.matmul(z[off:off + m], M, out=x[off:off + m])
            x[off:off + m] += means[c] * w[off:off + m, None].sqrt()
        off += m
    x /= w.sqrt()[:, None]
    return x.contiguous()


def _chi2_torch(n: int, nu: float, g, device):
    """Chi-squared(nu) draws as the sum of nu squared normals (integer nu) or
    a Gamma(nu/2, 2) draw otherwise."""
    import torch

    if float(nu).is_integer():
        z = torch.randn(n, int(nu), generator=g, device=device, dtype=torch.float64)
        return (z * z).sum(1)
    return torch._standard_gamma(torch.full((n,), nu / 2.0, device=device, dtype=torch.float64)) * 2.0


def subsample(X: np.ndarray, n: int, seed: int = 0) -> np.ndarray:
    """Seeded row subsample (without replacement), rows kept in index order."""
    if n >= X.shape[0]:
        return X
    rng = _rng(seed)
    rows = np.sort(rng.choice(X.shape[0], size=n, replace=False))
    return np.ascontiguousarray(X[rows])
