"""FP64 reference of the learned-direction network (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg
use this module; it shares no code with the CUDA path. It restates, in plain
numpy FP64 (matrix products are library primitives, nothing is fused):

* the input features of a pair (the future-work direction dictionary of
  Conclusion and Future Work, in the form this library implements): centroid difference, the 8
  leading principal components scaled by sqrt(lambda), per-dimension union
  variances, scaled by s = sqrt(trace(C) / D) (variances by s^2);
* the network h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), z = h2 W3 + b3,
  u_j = z_j / ||z_j|| (4 directions);
* the loss 1 - (1/tau) log sum_j exp(tau (u_j . w)^2), tau = 10, against the
  unit witness direction w of the exact Hausdorff distance (Eq. 1), averaged
  over the batch, and its gradient by the chain rule;
* Adam (beta 0.9 / 0.999, eps 1e-8, bias-corrected);
* the counter-based initialisation: SplitMix64 (Steele, Lea, Flood 2014) in
  the counter layout of the oracle's power-iteration start vectors, layer l
  drawing from stream 100 + l, weights uniform on +-sqrt(6 / fan_in).
"""
from __future__ import annotations

import numpy as np

from . import directions, hausdorff, union_covariance

TAU = 10.0
HIDDEN = 256
NDIRS = 4
NPCS = 8

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_units(seed: int, stream: int, idx) -> np.ndarray:
    """Element i of stream l: state = seed + (l * 2^32 + i + 1) * golden
    (mod 2^64), SplitMix64-mixed, top 53 bits mapped to [-1, 1)."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        c = (np.uint64(stream) << np.uint64(32)) + idx
        z = np.uint64(seed) + (c + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0) * 2.0 - 1.0


def bf16_round(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even): keep the top 16 bits of
    the FP32 pattern after adding 0x7FFF plus the lowest kept bit."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def shapes(D: int) -> dict:
    return dict(n_in=10 * D, h=HIDDEN, n_out=NDIRS * D)


def init_params(D: int, seed: int) -> dict:
    """Initial parameters (FP32 values held in FP64 arrays)."""
    s = shapes(D)
    dims = [(s["n_in"], s["h"]), (s["h"], s["h"]), (s["h"], s["n_out"])]
    P = {}
    for layer, (fi, fo) in enumerate(dims, start=1):
        u = splitmix64_units(seed, 100 + layer, np.arange(fi * fo))
        P[f"W{layer}"] = (np.sqrt(6.0 / fi) * u).astype(np.float32).astype(np.float64).reshape(fi, fo)
        P[f"b{layer}"] = np.zeros(fo)
    return P


def forward(P: dict, X, W=None, bf16: bool = False) -> dict:
    """Forward pass of a batch X [B, 10D]; with labels W [B, D] also the loss
    per sample and its mean. bf16: every operand of a matrix product is
    rounded to BF16 first (the products and sums stay FP64), the arithmetic
    of the library's BF16 tensor-core path with its ReLU decisions taken on
    the same rounded operands."""
    R = bf16_round if bf16 else (lambda v: v)
    X = np.asarray(X, dtype=np.float64)
    B = X.shape[0]
    a1 = R(X) @ R(P["W1"]) + P["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = R(h1) @ R(P["W2"]) + P["b2"]
    h2 = np.maximum(a2, 0.0)
    z = R(h2) @ R(P["W3"]) + P["b3"]
    D = z.shape[1] // NDIRS
    Z = z.reshape(B, NDIRS, D)
    nrm = np.sqrt((Z * Z).sum(axis=2))
    U = Z / nrm[:, :, None]
    out = dict(X=X, a1=a1, h1=h1, a2=a2, h2=h2, z=z, Z=Z, nrm=nrm, U=U, bf16=bf16)
    if W is not None:
        W = np.asarray(W, dtype=np.float64)
        dot = np.einsum("bjd,bd->bj", U, W)
        c = dot * dot
        mx = (TAU * c).max(axis=1, keepdims=True)
        lse = mx[:, 0] + np.log(np.exp(TAU * c - mx).sum(axis=1))
        out.update(W=W, dot=dot, c=c, loss=1.0 - lse / TAU, p=np.exp(TAU * c - lse[:, None]))
        out["loss_mean"] = float(out["loss"].mean())
    return out


def backward(P: dict, f: dict) -> dict:
    """Gradient of the mean loss with respect to every parameter (chain rule,
    one step per operation of the forward pass)."""
    R = bf16_round if f.get("bf16") else (lambda v: v)
    B = f["X"].shape[0]
    U, W, dot, p, nrm = f["U"], f["W"], f["dot"], f["p"], f["nrm"]
    # d loss_b / d c_bj = -p_bj; c = dot^2 with dot = u . w; mean over B
    g_dot = -p * 2.0 * dot / B                                # d/d dot
    g_U = g_dot[:, :, None] * W[:, None, :]                   # d/d u_j
    # u = z / ||z||: dz = (g - (u . g) u) / ||z||
    ug = (U * g_U).sum(axis=2, keepdims=True)
    g_Z = (g_U - ug * U) / nrm[:, :, None]
    g_z = g_Z.reshape(B, -1)
    G = {}
    G["W3"] = R(f["h2"]).T @ R(g_z)
    G["b3"] = g_z.sum(axis=0)
    g_h2 = R(g_z) @ R(P["W3"]).T
    g_a2 = g_h2 * (f["a2"] > 0)
    G["W2"] = R(f["h1"]).T @ R(g_a2)
    G["b2"] = g_a2.sum(axis=0)
    g_h1 = R(g_a2) @ R(P["W2"]).T
    g_a1 = g_h1 * (f["a1"] > 0)
    G["W1"] = R(f["X"]).T @ R(g_a1)
    G["b1"] = g_a1.sum(axis=0)
    return G


def adam_step(P: dict, M: dict, V: dict, G: dict, lr: float, step: int,
              b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update in place (bias correction with 1 - b^step)."""
    c1, c2 = 1.0 - b1**step, 1.0 - b2**step
    for k in P:
        M[k] = b1 * M[k] + (1.0 - b1) * G[k]
        V[k] = b2 * V[k] + (1.0 - b2) * G[k] * G[k]
        P[k] = P[k] - lr * (M[k] / c1) / (np.sqrt(V[k] / c2) + eps)


def features(A, B, seed: int = 0) -> np.ndarray:
    """Input features [10 D] of a pair from the oracle's own directions."""
    A = np.asarray(A, dtype=np.float32)
    B = np.asarray(B, dtype=np.float32)
    D = A.shape[1]
    dirs, lam, _ = directions(A, B, m=NPCS, seed=seed)
    _, C = union_covariance(A, B)
    dmu = B.astype(np.float64).mean(0) - A.astype(np.float64).mean(0)
    var = np.diag(C).copy()
    s2 = var.sum() / D if var.sum() > 0 else 1.0
    s = np.sqrt(s2)
    pcs = np.sqrt(np.maximum(lam, 0.0))[:, None] * dirs[1:1 + NPCS]
    return np.concatenate([dmu / s, pcs.reshape(-1) / s, var / s2])


def witness_direction(A, B) -> np.ndarray:
    """Unit vector (a* - b*)/||a* - b*|| of the exact HD's witness pair."""
    r = hausdorff(A, B)
    d = np.asarray(A[r["wit_a"]], dtype=np.float64) - np.asarray(B[r["wit_b"]], dtype=np.float64)
    n = np.linalg.norm(d)
    return d / n if n > 0 else d


def flatten(P: dict, D: int) -> np.ndarray:
    """Parameters in the library's layout: W1, b1, W2, b2, W3, b3, each
    row-major and padded to a multiple of 64 floats."""
    parts = []
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        v = np.asarray(P[k], dtype=np.float64).reshape(-1)
        pad = (-v.size) % 64
        parts.append(np.concatenate([v, np.zeros(pad)]))
    return np.concatenate(parts)


def unflatten(flat, D: int) -> dict:
    s = shapes(D)
    dims = {"W1": (s["n_in"], s["h"]), "b1": (s["h"],), "W2": (s["h"], s["h"]), "b2": (s["h"],),
            "W3": (s["h"], s["n_out"]), "b3": (s["n_out"],)}
    P, o = {}, 0
    flat = np.asarray(flat, dtype=np.float64)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        n = int(np.prod(dims[k]))
        P[k] = flat[o:o + n].reshape(dims[k]).copy()
        o += n + ((-n) % 64)
    return P
