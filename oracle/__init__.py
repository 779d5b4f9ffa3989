"""FP64 CPU oracle for ProHD (arxiv 2511.18207).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code with
the CUDA library (``paper_2511_18207_gb300``) and never imports it.

The arithmetic lives in ``prohd_oracle.c`` (plain C, FP64, no FMA contraction).
This module compiles it on first use, loads it with ctypes and composes the
paper's Algorithm 3 (ProjHausdorff) from its pieces:

* ``directed_hd`` / ``hausdorff``   Eq. 1, brute force
* ``directions``                    Algorithm 1 (centroid axis) + Algorithm 2
                                    (top-m principal components of [A; B])
* ``select``                        Algorithms 1-2 (bottom-k / top-k, union)
* ``prohd``                         Algorithm 3
* ``hd_1d`` / ``delta``             the quantities of the bounds in Methodology – Theoretical Properties
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "prohd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libprohd_oracle.so")

#: gcc flags: keep every FP64 operation separately rounded.
CFLAGS = ["-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp", "-std=c11"]

_lock = threading.Lock()
_lib = None


def build_oracle(force: bool = False) -> str:
    """Compile ``prohd_oracle.c`` into ``_build/libprohd_oracle.so``."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build_oracle())
        f32p = ctypes.POINTER(ctypes.c_float)
        f64p = ctypes.POINTER(ctypes.c_double)
        i64p = ctypes.POINTER(ctypes.c_int64)
        i64 = ctypes.c_int64
        lib.oracle_directed_hd.argtypes = [f32p, i64, f32p, i64, ctypes.c_int, i64, i64,
                                           f64p, i64p, i64p, f64p, i64p]
        lib.oracle_directed_hd.restype = ctypes.c_int
        lib.oracle_centroid.argtypes = [f32p, i64, ctypes.c_int, f64p]
        lib.oracle_centroid_axis.argtypes = [f64p, f64p, ctypes.c_int, f64p]
        lib.oracle_union_covariance.argtypes = [f32p, i64, f32p, i64, ctypes.c_int, f64p, f64p]
        lib.oracle_splitmix64_unit.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_splitmix64_unit.restype = ctypes.c_double
        lib.oracle_power_iteration.argtypes = [f64p, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                               ctypes.c_double, ctypes.c_int, f64p, f64p,
                                               ctypes.POINTER(ctypes.c_int)]
        lib.oracle_power_iteration.restype = ctypes.c_int
        lib.oracle_project.argtypes = [f32p, i64, ctypes.c_int, f64p, f64p]
        lib.oracle_k_of.argtypes = [ctypes.c_double, i64]
        lib.oracle_k_of.restype = i64
        lib.oracle_select.argtypes = [f32p, i64, ctypes.c_int, f64p, ctypes.c_int, i64p,
                                      ctypes.POINTER(ctypes.c_uint8)]
        lib.oracle_select.restype = ctypes.c_int
        lib.oracle_hd_1d.argtypes = [f64p, i64, f64p, i64]
        lib.oracle_hd_1d.restype = ctypes.c_double
        lib.oracle_delta.argtypes = [f32p, i64, ctypes.c_int, f64p]
        lib.oracle_delta.restype = ctypes.c_double
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _f32(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    if x.ndim != 2:
        raise ValueError("point sets are [n, D] arrays")
    return x


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def num_threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_num_threads())


# --------------------------------------------------------------------------
# Eq. 1: exact Hausdorff distance
# --------------------------------------------------------------------------

def directed_hd(X, Y, row_begin: int = 0, row_end: int | None = None, want_rows: bool = False):
    """h(X, Y) over the outer rows [row_begin, row_end) (Eq. 1), FP64.

    Returns (h, i, j) with the witness pair (lowest indices on ties); with
    ``want_rows`` also the per-row squared NN distances and NN indices.
    """
    lib = _load()
    X, Y = _f32(X), _f32(Y)
    if X.shape[1] != Y.shape[1]:
        raise ValueError("dimension mismatch")
    nX, D = X.shape
    nY = Y.shape[0]
    if row_end is None:
        row_end = nX
    h = ctypes.c_double()
    i = ctypes.c_int64()
    j = ctypes.c_int64()
    rm = np.full(nX, np.nan) if want_rows else None
    ra = np.full(nX, -1, dtype=np.int64) if want_rows else None
    rc = lib.oracle_directed_hd(_p(X, ctypes.c_float), nX, _p(Y, ctypes.c_float), nY, D,
                                row_begin, row_end, ctypes.byref(h), ctypes.byref(i), ctypes.byref(j),
                                _p(rm, ctypes.c_double) if want_rows else None,
                                _p(ra, ctypes.c_int64) if want_rows else None)
    if rc != 0:
        raise ValueError("oracle_directed_hd: bad arguments")
    if want_rows:
        return h.value, i.value, j.value, rm, ra
    return h.value, i.value, j.value


def hausdorff(A, B):
    """Symmetric HD H(A,B) = max(h(A,B), h(B,A)) (Eq. 1), FP64.

    Returns a dict: H, h_ab, h_ba, witness (a index, b index) of H, dir (0 if
    h(A,B) >= h(B,A) else 1)."""
    h_ab, ia, jb = directed_hd(A, B)
    h_ba, jb2, ia2 = directed_hd(B, A)
    if h_ab >= h_ba:
        return dict(H=h_ab, h_ab=h_ab, h_ba=h_ba, wit_a=ia, wit_b=jb, dir=0)
    return dict(H=h_ba, h_ab=h_ab, h_ba=h_ba, wit_a=ia2, wit_b=jb2, dir=1)


# --------------------------------------------------------------------------
# Algorithms 1-2: directions
# --------------------------------------------------------------------------

def centroid(X) -> np.ndarray:
    lib = _load()
    X = _f32(X)
    out = np.zeros(X.shape[1])
    lib.oracle_centroid(_p(X, ctypes.c_float), X.shape[0], X.shape[1], _p(out, ctypes.c_double))
    return out


def centroid_axis(xbar, ybar) -> np.ndarray:
    lib = _load()
    xbar = np.ascontiguousarray(xbar, dtype=np.float64)
    ybar = np.ascontiguousarray(ybar, dtype=np.float64)
    u = np.zeros_like(xbar)
    lib.oracle_centroid_axis(_p(xbar, ctypes.c_double), _p(ybar, ctypes.c_double), xbar.size,
                             _p(u, ctypes.c_double))
    return u


def union_covariance(A, B):
    """(mu, C) of the stacked set [A; B], two-pass FP64 (Algorithm 2)."""
    lib = _load()
    A, B = _f32(A), _f32(B)
    D = A.shape[1]
    mu = np.zeros(D)
    C = np.zeros((D, D))
    lib.oracle_union_covariance(_p(A, ctypes.c_float), A.shape[0], _p(B, ctypes.c_float), B.shape[0], D,
                                _p(mu, ctypes.c_double), _p(C, ctypes.c_double))
    return mu, C


def splitmix64_unit(seed: int, l: int, j: int) -> float:
    return float(_load().oracle_splitmix64_unit(seed, l, j))


def power_iteration(C, m: int, seed: int = 0, tol: float = 1e-13, maxit: int = 1000):
    """Top-m eigenpairs of C by deflated power iteration. Returns (U [m,D], lam [m], iters [m])."""
    lib = _load()
    C = np.ascontiguousarray(C, dtype=np.float64)
    D = C.shape[0]
    U = np.zeros((m, D))
    lam = np.zeros(m)
    it = np.zeros(m, dtype=np.int32)
    rc = lib.oracle_power_iteration(_p(C, ctypes.c_double), D, m, seed, tol, maxit,
                                    _p(U, ctypes.c_double), _p(lam, ctypes.c_double),
                                    _p(it, ctypes.c_int))
    if rc != 0:
        raise ValueError("oracle_power_iteration: bad arguments")
    return U, lam, it


def default_m(D: int) -> int:
    """m = floor(sqrt(D)) (Methodology – Background and Notation)."""
    return int(math.isqrt(D))


def directions(A, B, m: int | None = None, seed: int = 0, tol: float = 1e-13, maxit: int = 1000):
    """Direction list [u0 (centroid axis); u1..um (PCs)] as an [1+m, D] FP64 array,
    with the PCs' eigenvalues and iteration counts."""
    A, B = _f32(A), _f32(B)
    D = A.shape[1]
    if m is None:
        m = default_m(D)
    u0 = centroid_axis(centroid(A), centroid(B))
    _, C = union_covariance(A, B)
    U, lam, it = power_iteration(C, m, seed, tol, maxit)
    return np.vstack([u0[None, :], U]), lam, it


# --------------------------------------------------------------------------
# Algorithms 1-2: selection
# --------------------------------------------------------------------------

def k_of(alpha: float, n: int) -> int:
    """k = max(1, floor(alpha n)), clamped to n."""
    return int(_load().oracle_k_of(float(alpha), int(n)))


def project(X, u) -> np.ndarray:
    lib = _load()
    X = _f32(X)
    u = np.ascontiguousarray(u, dtype=np.float64)
    p = np.zeros(X.shape[0])
    lib.oracle_project(_p(X, ctypes.c_float), X.shape[0], X.shape[1], _p(u, ctypes.c_double),
                       _p(p, ctypes.c_double))
    return p


def select_mask(X, dirs, k_per_dir) -> np.ndarray:
    """Union over directions of the bottom-k and top-k points; uint8 mask [n]."""
    lib = _load()
    X = _f32(X)
    dirs = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    k = np.ascontiguousarray(k_per_dir, dtype=np.int64)
    if dirs.shape[1] != X.shape[1] or k.size != dirs.shape[0]:
        raise ValueError("shape mismatch")
    mask = np.zeros(X.shape[0], dtype=np.uint8)
    rc = lib.oracle_select(_p(X, ctypes.c_float), X.shape[0], X.shape[1], _p(dirs, ctypes.c_double),
                           dirs.shape[0], _p(k, ctypes.c_int64), _p(mask, ctypes.c_uint8))
    if rc != 0:
        raise ValueError("oracle_select failed")
    return mask


def select(X, dirs, k_per_dir) -> np.ndarray:
    """Sorted unique indices of the selected points (int64)."""
    return np.flatnonzero(select_mask(X, dirs, k_per_dir)).astype(np.int64)


def k_list(n: int, nd: int, alpha_c: float, alpha_p: float):
    """Per-direction k: k_c for the centroid axis, k_p for each PC (Algorithm 3)."""
    return [k_of(alpha_c, n)] + [k_of(alpha_p, n)] * (nd - 1)


# --------------------------------------------------------------------------
# Algorithm 3
# --------------------------------------------------------------------------

def prohd(A, B, alpha: float = 0.01, m: int | None = None, alpha_p: float | None = None,
          seed: int = 0, tol: float = 1e-13, maxit: int = 1000, dirs=None):
    """ProjHausdorff (Algorithm 3).

    m defaults to floor(sqrt(D)) and alpha_p to alpha / m. ``dirs`` (an
    [nd, D] FP64 array whose first row is the centroid axis) replaces the
    computed directions when given. Returns a dict with H_hat, h_ab, h_ba,
    idxA, idxB (sorted unique), dirs, lam, and the witness of H_hat in the
    original index space."""
    A, B = _f32(A), _f32(B)
    D = A.shape[1]
    lam = None
    if dirs is None:
        if m is None:
            m = default_m(D)
        dirs, lam, _ = directions(A, B, m=m, seed=seed, tol=tol, maxit=maxit)
    nd = dirs.shape[0]
    mm = max(nd - 1, 1)
    if alpha_p is None:
        alpha_p = alpha / mm
    idxA = select(A, dirs, k_list(A.shape[0], nd, alpha, alpha_p))
    idxB = select(B, dirs, k_list(B.shape[0], nd, alpha, alpha_p))
    r = hausdorff(A[idxA], B[idxB])
    return dict(H_hat=r["H"], h_ab=r["h_ab"], h_ba=r["h_ba"], dir=r["dir"],
                wit_a=int(idxA[r["wit_a"]]), wit_b=int(idxB[r["wit_b"]]),
                idxA=idxA, idxB=idxB, dirs=dirs, lam=lam)


def refined(A, B, idxA, idxB):
    """One-sided refinement of a ProHD estimate (reading of the Theoretical Properties subsection's
    underestimation claim): max(h(A_sel, B), h(B_sel, A)), each selected
    point's nearest neighbour searched in the whole other set. Every term is
    a true nearest-neighbour distance of a point of A (or B), so the result
    never exceeds H(A, B) (Eq. 1). Returns a dict with H1, h_ab, h_ba, dir and
    the witness of H1 in the original index space."""
    A, B = _f32(A), _f32(B)
    idxA = np.asarray(idxA, dtype=np.int64)
    idxB = np.asarray(idxB, dtype=np.int64)
    h_ab, ia, jb = directed_hd(A[idxA], B)
    h_ba, jb2, ia2 = directed_hd(B[idxB], A)
    if h_ab >= h_ba:
        return dict(H1=h_ab, h_ab=h_ab, h_ba=h_ba, dir=0, wit_a=int(idxA[ia]), wit_b=int(jb))
    return dict(H1=h_ba, h_ab=h_ab, h_ba=h_ba, dir=1, wit_a=int(ia2), wit_b=int(idxB[jb2]))


ADAPTIVE_MAX_STEPS = 32


def adaptive(A, B, alpha: float, alpha_max: float, rel_tol: float, m: int | None = None,
             alpha_p: float | None = None, seed: int = 0, dirs=None, max_steps: int = ADAPTIVE_MAX_STEPS):
    """Adaptive alpha schedule (the future direction of Conclusion and Future Work: alpha grown
    until the estimate meets an error budget), read as a doubling schedule on
    the one-sided refined estimate.

    Directions are taken once (or given). Step t keeps alpha_t = alpha 2^t on
    the centroid axis and alpha_p 2^t on each component (alpha_p defaults to
    alpha / m), selects as Algorithm 3 does, and takes the refined estimate
    H_t = max(h(A_sel, B), h(B_sel, A)). Candidate sets grow with t, so H_t
    never decreases and never exceeds H. The schedule stops, checked in this
    order, when every point is selected on both sides (H_t = H), when t >= 1
    and H_t - H_{t-1} <= rel_tol H_t, when alpha 2^(t+1) > alpha_max, or after
    ``max_steps`` steps. Returns H1 (the last H_t), the per-step H and subset
    sizes, the number of steps, the stop reason and the last alpha values."""
    A, B = _f32(A), _f32(B)
    D = A.shape[1]
    if dirs is None:
        if m is None:
            m = default_m(D)
        dirs, _, _ = directions(A, B, m=m, seed=seed)
    dirs = np.atleast_2d(np.asarray(dirs, dtype=np.float64))
    nd = dirs.shape[0]
    if alpha_p is None:
        alpha_p = alpha / max(nd - 1, 1)
    Hs, na, nb = [], [], []
    t = 0
    while True:
        a_t, ap_t = alpha * 2.0**t, alpha_p * 2.0**t
        ia = select(A, dirs, k_list(A.shape[0], nd, a_t, ap_t))
        ib = select(B, dirs, k_list(B.shape[0], nd, a_t, ap_t))
        r = refined(A, B, ia, ib)
        Hs.append(r["H1"])
        na.append(int(ia.size))
        nb.append(int(ib.size))
        if ia.size == A.shape[0] and ib.size == B.shape[0]:
            reason = "all"
        elif t >= 1 and Hs[-1] - Hs[-2] <= rel_tol * Hs[-1]:
            reason = "stable"
        elif alpha * 2.0 ** (t + 1) > alpha_max:
            reason = "budget"
        elif t + 1 >= max_steps:
            reason = "steps"
        else:
            t += 1
            continue
        return dict(H1=Hs[-1], H=Hs, nsel_a=na, nsel_b=nb, steps=t + 1, reason=reason, alpha=a_t, alpha_p=ap_t,
                    idxA=ia, idxB=ib, refined=r, dirs=dirs)


# --------------------------------------------------------------------------
# Methodology – Theoretical Properties quantities
# --------------------------------------------------------------------------

def hd_1d(pX, pY) -> float:
    """1D directed HD max_i min_j |pX_i - pY_j|."""
    lib = _load()
    pX = np.ascontiguousarray(pX, dtype=np.float64)
    pY = np.ascontiguousarray(pY, dtype=np.float64)
    return float(lib.oracle_hd_1d(_p(pX, ctypes.c_double), pX.size, _p(pY, ctypes.c_double), pY.size))


def H_u(A, B, u) -> float:
    """H_u(A,B) = max(h_u(A,B), h_u(B,A)) along the unit direction u."""
    pA, pB = project(A, u), project(B, u)
    return max(hd_1d(pA, pB), hd_1d(pB, pA))


def delta(A, B, u) -> float:
    """delta(u) over A union B (Eq. 2)."""
    lib = _load()
    A, B = _f32(A), _f32(B)
    u = np.ascontiguousarray(u, dtype=np.float64)
    dA = lib.oracle_delta(_p(A, ctypes.c_float), A.shape[0], A.shape[1], _p(u, ctypes.c_double))
    dB = lib.oracle_delta(_p(B, ctypes.c_float), B.shape[0], B.shape[1], _p(u, ctypes.c_double))
    return float(max(dA, dB))
