"""Thin Python binding of the ProHD C ABI (``include/prohd.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library ``_lib/libprohd.so``. PyTorch provides device memory (inputs,
workspaces, result buffers) and streams. There is no fallback: if the library
is missing or the GPU is not an sm_103 device, calls raise.

Low-level calls mirror the C names (``hausdorff_exact``, ``prohd_directions``,
``prohd_select``, ``prohd_estimate``, ``prohd_estimate_host``) and enqueue on
the current torch stream without synchronising; the ``*_sync`` helpers wait and
decode the device result into a dict.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libprohd.so")

PROHD_OK, PROHD_EINVAL, PROHD_ENOMEM, PROHD_ECUDA, PROHD_ETIMEOUT, PROHD_ENONFINITE, PROHD_ENOTSUP = range(7)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENONFINITE", 6: "ENOTSUP"}
PRECISIONS = {"fp32": 0, "fp16": 1, "bf16": 2}

#: every symbol include/prohd.h declares
EXPORTS = [
    "prohd_create", "prohd_destroy", "prohd_last_error", "prohd_params_default", "prohd_k_of",
    "hausdorff_exact_workspace_size", "prohd_directions_workspace_size", "prohd_select_workspace_size",
    "prohd_estimate_workspace_size", "prohd_estimate_host_workspace_size",
    "hausdorff_exact", "prohd_directions", "prohd_select", "prohd_estimate", "prohd_estimate_host",
    "prohd_profile_enable", "prohd_profile_read", "prohd_launch_count", "hausdorff_exact_noalloc",
    "prohd_batch_workspace_size", "prohd_batch_plan", "prohd_batch_destroy", "prohd_estimate_batched",
    "prohd_batch_use_graph", "prohd_batch_autotune", "prohd_batch_get_tunables", "prohd_batch_set_tunables",
    "prohd_batch_pair_outputs", "prohd_tunables_save", "prohd_tunables_load",
    "prohd_estimate_dirs_workspace_size", "prohd_estimate_dirs", "prohd_features_workspace_size", "prohd_features",
    "prohd_mlp_param_count", "prohd_mlp_state_bytes", "prohd_mlp_scratch_bytes", "prohd_mlp_init", "prohd_mlp_forward",
    "prohd_mlp_loss_grad", "prohd_mlp_train_step", "prohd_mlp_adam_step",
    "prohd_estimate_adaptive_workspace_size", "prohd_estimate_adaptive",
    "hausdorff_exact_pruned_workspace_size", "hausdorff_exact_pruned", "prohd_set_prune_min_pairs",
    "prohd_set_subset_prune_min_pairs",
    "prohd_covariance_workspace_size", "prohd_covariance", "prohd_mlp_save", "prohd_mlp_load",
]

#: prohd_phase names, in enum order
PHASES = ["gram", "power", "project", "select", "gather", "hd_prep", "hd_contract", "hd_rescore"]


class Params(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("precision", ctypes.c_int32), ("alpha_c", ctypes.c_double),
                ("alpha_p", ctypes.c_double), ("power_max_iters", ctypes.c_int32), ("refine", ctypes.c_int32),
                ("power_tol", ctypes.c_double), ("seed", ctypes.c_uint64), ("wait_timeout_ns", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 4)]


class HdResult(ctypes.Structure):
    _fields_ = [("H", ctypes.c_double), ("h_ab", ctypes.c_double), ("h_ba", ctypes.c_double),
                ("wit_a", ctypes.c_int64), ("wit_b", ctypes.c_int64), ("ab_a", ctypes.c_int64),
                ("ab_b", ctypes.c_int64), ("ba_b", ctypes.c_int64), ("ba_a", ctypes.c_int64),
                ("dir", ctypes.c_int32), ("status", ctypes.c_int32), ("H_lowp", ctypes.c_double),
                ("n_rescored_a", ctypes.c_int64), ("n_rescored_b", ctypes.c_int64)]


class Result(ctypes.Structure):
    _fields_ = [("hd", HdResult), ("nsel_a", ctypes.c_int64), ("nsel_b", ctypes.c_int64)]


ADAPT_MAX_STEPS = 32
ADAPT_REASONS = {0: "all", 1: "stable", 2: "budget", 3: "steps"}


class AdaptiveInfo(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int32), ("reason", ctypes.c_int32), ("alpha_c", ctypes.c_double),
                ("alpha_p", ctypes.c_double), ("H", ctypes.c_double * ADAPT_MAX_STEPS),
                ("nsel_a", ctypes.c_int64 * ADAPT_MAX_STEPS), ("nsel_b", ctypes.c_int64 * ADAPT_MAX_STEPS)]


class PairDesc(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("nA", ctypes.c_int64), ("B", ctypes.c_void_p), ("nB", ctypes.c_int64),
                ("D", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None
_lib_lock = threading.Lock()


def load_library(path: str = LIB_PATH):
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise FileNotFoundError(f"{path} is missing: build it with __graft_entry__.build() "
                                    "or python -m paper_2511_18207_gb300.build_lib")
        lib = ctypes.CDLL(path)
        vp, i64, i32, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t
        pp = ctypes.POINTER(Params)
        lib.prohd_create.argtypes = [ctypes.POINTER(vp)]
        lib.prohd_create.restype = i32
        lib.prohd_destroy.argtypes = [vp]
        lib.prohd_destroy.restype = None
        lib.prohd_last_error.argtypes = [vp]
        lib.prohd_last_error.restype = ctypes.c_char_p
        lib.prohd_params_default.argtypes = [pp]
        lib.prohd_params_default.restype = None
        lib.prohd_k_of.argtypes = [ctypes.c_double, i64]
        lib.prohd_k_of.restype = i64
        lib.hausdorff_exact_workspace_size.argtypes = [i64, i64, i32, i32]
        lib.hausdorff_exact_workspace_size.restype = sz
        lib.prohd_directions_workspace_size.argtypes = [i64, i64, i32, i32]
        lib.prohd_directions_workspace_size.restype = sz
        lib.prohd_select_workspace_size.argtypes = [i64, i64, i32, i32]
        lib.prohd_select_workspace_size.restype = sz
        lib.prohd_estimate_workspace_size.argtypes = [i64, i64, i32, pp]
        lib.prohd_estimate_workspace_size.restype = sz
        lib.prohd_estimate_host_workspace_size.argtypes = [i64, i64, i32, pp]
        lib.prohd_estimate_host_workspace_size.restype = sz
        lib.hausdorff_exact.argtypes = [vp, vp, i64, vp, i64, i32, i32, vp, vp, sz, vp]
        lib.hausdorff_exact.restype = i32
        lib.prohd_directions.argtypes = [vp, vp, i64, vp, i64, i32, pp, vp, vp, vp, sz, vp]
        lib.prohd_directions.restype = i32
        lib.prohd_mlp_save.argtypes = [vp, ctypes.c_char_p, i32, i64, vp, vp, i64, vp]
        lib.prohd_mlp_save.restype = i32
        lib.prohd_mlp_load.argtypes = [vp, ctypes.c_char_p, ctypes.POINTER(i32), ctypes.POINTER(i64), vp, vp, i64,
                                       ctypes.POINTER(i64), vp]
        lib.prohd_mlp_load.restype = i32
        lib.prohd_covariance_workspace_size.argtypes = [i64, i64, i32]
        lib.prohd_covariance_workspace_size.restype = sz
        lib.prohd_covariance.argtypes = [vp, vp, i64, vp, i64, i32, vp, vp, vp, sz, vp]
        lib.prohd_covariance.restype = i32
        lib.prohd_select.argtypes = [vp, vp, i64, vp, i64, i32, vp, i32, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        lib.prohd_select.restype = i32
        lib.prohd_estimate.argtypes = [vp, vp, i64, vp, i64, i32, pp, vp, vp, vp, vp, vp, sz, vp]
        lib.prohd_estimate.restype = i32
        lib.prohd_estimate_host.argtypes = [vp, vp, i64, vp, i64, i32, pp, vp, vp, sz, vp]
        lib.prohd_estimate_host.restype = i32
        lib.prohd_profile_enable.argtypes = [vp, i32]
        lib.prohd_profile_enable.restype = i32
        lib.prohd_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64), i32]
        lib.prohd_profile_read.restype = i32
        lib.prohd_launch_count.argtypes = []
        lib.prohd_launch_count.restype = ctypes.c_uint64
        lib.hausdorff_exact_noalloc.argtypes = [vp, vp, i64, vp, i64, i32, vp, vp]
        lib.hausdorff_exact_noalloc.restype = i32
        pd = ctypes.POINTER(PairDesc)
        pi32 = ctypes.POINTER(ctypes.c_int32)
        lib.prohd_batch_workspace_size.argtypes = [pd, i32, pp]
        lib.prohd_batch_workspace_size.restype = sz
        lib.prohd_batch_plan.argtypes = [vp, pd, i32, pp, vp, sz, ctypes.POINTER(vp)]
        lib.prohd_batch_plan.restype = i32
        lib.prohd_batch_destroy.argtypes = [vp]
        lib.prohd_batch_destroy.restype = None
        lib.prohd_estimate_batched.argtypes = [vp, vp, vp, vp]
        lib.prohd_estimate_batched.restype = i32
        lib.prohd_batch_use_graph.argtypes = [vp, i32]
        lib.prohd_batch_use_graph.restype = i32
        lib.prohd_batch_autotune.argtypes = [vp, vp, vp, vp, ctypes.POINTER(ctypes.c_double)]
        lib.prohd_batch_autotune.restype = i32
        lib.prohd_batch_get_tunables.argtypes = [vp, pi32, pi32, pi32]
        lib.prohd_batch_get_tunables.restype = i32
        lib.prohd_batch_set_tunables.argtypes = [vp, i32, i32, i32]
        lib.prohd_batch_set_tunables.restype = i32
        lib.prohd_batch_pair_outputs.argtypes = [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                 ctypes.POINTER(vp)]
        lib.prohd_batch_pair_outputs.restype = i32
        pi64 = ctypes.POINTER(ctypes.c_int64)
        lib.prohd_estimate_dirs_workspace_size.argtypes = [i64, i64, i32, i32, pi64, pi64, pp]
        lib.prohd_estimate_dirs_workspace_size.restype = sz
        lib.prohd_estimate_dirs.argtypes = [vp, vp, i64, vp, i64, i32, pp, vp, i32, pi64, pi64, vp, vp, vp, vp, sz, vp]
        lib.prohd_estimate_dirs.restype = i32
        lib.hausdorff_exact_pruned_workspace_size.argtypes = [i64, i64, i32, i32]
        lib.hausdorff_exact_pruned_workspace_size.restype = sz
        lib.hausdorff_exact_pruned.argtypes = [vp, vp, i64, vp, i64, i32, i32, vp, pi64, vp, sz, vp]
        lib.hausdorff_exact_pruned.restype = i32
        lib.prohd_set_prune_min_pairs.argtypes = [vp, ctypes.c_double]
        lib.prohd_set_prune_min_pairs.restype = i32
        lib.prohd_set_subset_prune_min_pairs.argtypes = [vp, ctypes.c_double]
        lib.prohd_set_subset_prune_min_pairs.restype = i32
        lib.prohd_tunables_save.argtypes = [vp, ctypes.c_char_p]
        lib.prohd_tunables_save.restype = i32
        lib.prohd_tunables_load.argtypes = [vp, ctypes.c_char_p]
        lib.prohd_tunables_load.restype = i32
        lib.prohd_estimate_adaptive_workspace_size.argtypes = [i64, i64, i32, pp, ctypes.c_double]
        lib.prohd_estimate_adaptive_workspace_size.restype = sz
        lib.prohd_estimate_adaptive.argtypes = [vp, vp, i64, vp, i64, i32, pp, ctypes.c_double, ctypes.c_double, vp,
                                                ctypes.POINTER(AdaptiveInfo), vp, vp, vp, vp, sz, vp]
        lib.prohd_estimate_adaptive.restype = i32
        lib.prohd_features_workspace_size.argtypes = [i64, i64, i32]
        lib.prohd_features_workspace_size.restype = sz
        lib.prohd_features.argtypes = [vp, vp, i64, vp, i64, i32, pp, vp, vp, vp, vp, sz, vp]
        lib.prohd_features.restype = i32
        for f in ("prohd_mlp_param_count", "prohd_mlp_state_bytes"):
            getattr(lib, f).argtypes = [i32]
            getattr(lib, f).restype = sz
        lib.prohd_mlp_scratch_bytes.argtypes = [i32, i32]
        lib.prohd_mlp_scratch_bytes.restype = sz
        lib.prohd_mlp_init.argtypes = [vp, i32, ctypes.c_uint64, vp, vp]
        lib.prohd_mlp_init.restype = i32
        lib.prohd_mlp_forward.argtypes = [vp, i32, vp, vp, i32, i32, vp, vp, vp, sz, vp]
        lib.prohd_mlp_forward.restype = i32
        lib.prohd_mlp_loss_grad.argtypes = [vp, i32, vp, vp, vp, i32, i32, vp, vp, vp, sz, vp]
        lib.prohd_mlp_loss_grad.restype = i32
        lib.prohd_mlp_train_step.argtypes = [vp, i32, vp, vp, vp, i32, i32, ctypes.c_float, i64, vp, vp, sz, vp]
        lib.prohd_mlp_train_step.restype = i32
        lib.prohd_mlp_adam_step.argtypes = [vp, i32, vp, vp, ctypes.c_float, i64, vp]
        lib.prohd_mlp_adam_step.restype = i32
        _lib = lib
        return lib


class ProHDError(RuntimeError):
    pass


def default_params(**kw) -> Params:
    p = Params()
    load_library().prohd_params_default(ctypes.byref(p))
    for k, v in kw.items():
        if v is None:
            continue
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        setattr(p, k, v)
    return p


def k_of(alpha: float, n: int) -> int:
    return int(load_library().prohd_k_of(float(alpha), int(n)))


def _torch():
    import torch
    return torch


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _check_points(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.device.type != "cuda" or t.dtype != torch.float32 or t.dim() != 2:
        raise ValueError(f"{name} must be a CUDA float32 tensor [n, D]")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Context:
    """Owns a prohd_ctx and a grow-only workspace on the current device."""

    def __init__(self):
        torch = _torch()
        lib = load_library()
        torch.cuda.init()
        h = ctypes.c_void_p()
        rc = lib.prohd_create(ctypes.byref(h))
        if rc != PROHD_OK:
            raise ProHDError(f"prohd_create failed: {STATUS_NAMES.get(rc, rc)} (the library needs an sm_103 GPU)")
        self.lib, self.h = lib, h
        self.device = torch.cuda.current_device()
        self._ws = None

    def close(self):
        if self.h:
            self.lib.prohd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace(self, nbytes: int):
        torch = _torch()
        nbytes = max(int(nbytes), 256)
        if self._ws is None or self._ws.numel() < nbytes:
            self._ws = torch.empty(nbytes, dtype=torch.uint8, device=f"cuda:{self.device}")
        return self._ws

    def _raise(self, rc, what):
        if rc != PROHD_OK:
            msg = self.lib.prohd_last_error(self.h).decode()
            raise ProHDError(f"{what}: {STATUS_NAMES.get(rc, rc)}: {msg}")

    @staticmethod
    def _stream(stream):
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream()
        return ctypes.c_void_p(s.cuda_stream)

    # ------------------------------------------------------------- profiling

    def profile_enable(self, on: bool = True):
        self._raise(self.lib.prohd_profile_enable(self.h, 1 if on else 0), "prohd_profile_enable")

    def profile_read(self, reset: bool = True) -> dict:
        """{phase: (total ms, instances)} of the calls made while profiling was on."""
        n = len(PHASES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        self._raise(self.lib.prohd_profile_read(self.h, ms, cnt, 1 if reset else 0), "prohd_profile_read")
        return {PHASES[i]: (ms[i], cnt[i]) for i in range(n)}

    def launch_count(self) -> int:
        return int(self.lib.prohd_launch_count())

    # ------------------------------------------------------------- C ABI mirrors

    def hausdorff_exact(self, A, B, precision="fp16", out=None, ws=None, stream=None):
        """Enqueues hausdorff_exact; returns the device result buffer (uint8 tensor)."""
        torch = _torch()
        _check_points(A, "A")
        _check_points(B, "B")
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        D = A.shape[1]
        need = self.lib.hausdorff_exact_workspace_size(A.shape[0], B.shape[0], D, prec)
        ws = self.workspace(need) if ws is None else ws
        out = torch.empty(ctypes.sizeof(HdResult), dtype=torch.uint8, device=A.device) if out is None else out
        rc = self.lib.hausdorff_exact(self.h, _ptr(A), A.shape[0], _ptr(B), B.shape[0], D, prec, _ptr(out),
                                      _ptr(ws), ws.numel(), self._stream(stream))
        self._raise(rc, "hausdorff_exact")
        return out

    def hausdorff_exact_pruned(self, A, B, precision="fp16", out=None, ws=None, stream=None, want_kept=False):
        """Enqueues hausdorff_exact_pruned; returns the device result buffer
        (and, with want_kept, the rows left per direction; that synchronises)."""
        torch = _torch()
        _check_points(A, "A")
        _check_points(B, "B")
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        D = A.shape[1]
        need = self.lib.hausdorff_exact_pruned_workspace_size(A.shape[0], B.shape[0], D, prec)
        ws = self.workspace(need) if ws is None else ws
        out = torch.empty(ctypes.sizeof(HdResult), dtype=torch.uint8, device=A.device) if out is None else out
        kept = (ctypes.c_int64 * 2)(-1, -1)
        rc = self.lib.hausdorff_exact_pruned(self.h, _ptr(A), A.shape[0], _ptr(B), B.shape[0], D, prec, _ptr(out),
                                             kept if want_kept else None, _ptr(ws), ws.numel(), self._stream(stream))
        self._raise(rc, "hausdorff_exact_pruned")
        return (out, [kept[0], kept[1]]) if want_kept else out

    def set_prune_min_pairs(self, min_pairs: float):
        """Pair threshold of the row pruning (pruned exact distance and the
        refinement); 0 prunes whenever the row counts allow."""
        self._raise(self.lib.prohd_set_prune_min_pairs(self.h, float(min_pairs)), "prohd_set_prune_min_pairs")

    def tunables_save(self, path: str):
        """Writes the context's batch item sizes to a tuning table file."""
        self._raise(self.lib.prohd_tunables_save(self.h, os.fsencode(path)), "prohd_tunables_save")

    def tunables_load(self, path: str):
        """Reads a tuning table file (of this device) into the context."""
        self._raise(self.lib.prohd_tunables_load(self.h, os.fsencode(path)), "prohd_tunables_load")

    def set_subset_prune_min_pairs(self, min_pairs: float):
        """Pair threshold of the estimate's pruned subset distance (same
        result as the plain contraction); 0 prunes whenever the subsets allow."""
        self._raise(self.lib.prohd_set_subset_prune_min_pairs(self.h, float(min_pairs)),
                    "prohd_set_subset_prune_min_pairs")

    def hausdorff_exact_noalloc(self, A, B, out=None, stream=None):
        """Enqueues hausdorff_exact_noalloc (FP32, library-internal scratch,
        no workspace); returns the device result buffer (uint8 tensor)."""
        torch = _torch()
        _check_points(A, "A")
        _check_points(B, "B")
        out = torch.empty(ctypes.sizeof(HdResult), dtype=torch.uint8, device=A.device) if out is None else out
        rc = self.lib.hausdorff_exact_noalloc(self.h, _ptr(A), A.shape[0], _ptr(B), B.shape[0], A.shape[1], _ptr(out),
                                              self._stream(stream))
        self._raise(rc, "hausdorff_exact_noalloc")
        return out

    def prohd_directions(self, A, B, m=None, seed=0, max_iters=None, tol=1e-13, stream=None):
        torch = _torch()
        _check_points(A, "A")
        _check_points(B, "B")
        D = A.shape[1]
        p = default_params(m=-1 if m is None else m, seed=seed, power_max_iters=max_iters, power_tol=tol)
        mm = int(math.isqrt(D)) if m is None else m
        dirs = torch.empty((1 + mm, D), dtype=torch.float64, device=A.device)
        eig = torch.empty(max(mm, 1), dtype=torch.float64, device=A.device)
        need = self.lib.prohd_directions_workspace_size(A.shape[0], B.shape[0], D, mm)
        ws = self.workspace(need)
        rc = self.lib.prohd_directions(self.h, _ptr(A), A.shape[0], _ptr(B), B.shape[0], D, ctypes.byref(p),
                                       _ptr(dirs), _ptr(eig), _ptr(ws), ws.numel(), self._stream(stream))
        self._raise(rc, "prohd_directions")
        return dirs, eig[:mm]

    def prohd_covariance(self, A, B, stream=None):
        """Union covariance C [D, D] and mean [D] of [A; B] (FP64 device tensors)."""
        torch = _torch()
        _check_points(A, "A")
        _check_points(B, "B")
        D = A.shape[1]
        C = torch.empty((D, D), dtype=torch.float64, device=A.device)
        mean = torch.empty(D, dtype=torch.float64, device=A.device)
        ws = self.workspace(self.lib.prohd_covariance_workspace_size(A.shape[0], B.shape[0], D))
        rc = self.lib.prohd_covariance(self.h, _ptr(A), A.shape[0], _ptr(B), B.shape[0], D, _ptr(C), _ptr(mean),
                                       _ptr(ws), ws.numel(), self._stream(stream))
        self._raise(rc, "prohd_covariance")
        return C, mean

    def prohd_select(self, A, B, dirs, kA, kB, stream=None):
        """Returns (idxA, nselA, idxB, nselB) device tensors (int32 indices, int64 counts)."""
        torch = _torch()
        _check_points(A, "A")
        _check_points(B, "B")
        D = A.shape[1]
        dirs = dirs.to(device=A.device, dtype=torch.float64).contiguous()
        nd = dirs.shape[0]
        ka = (ctypes.c_int64 * nd)(*[int(k) for k in kA])
        kb = (ctypes.c_int64 * nd)(*[int(k) for k in kB])
        idxA = torch.empty(A.shape[0], dtype=torch.int32, device=A.device)
        idxB = torch.empty(B.shape[0], dtype=torch.int32, device=A.device)
        ns = torch.zeros(2, dtype=torch.int64, device=A.device)
        need = self.lib.prohd_select_workspace_size(A.shape[0], B.shape[0], D, nd)
        ws = self.workspace(need)
        rc = self.lib.prohd_select(self.h, _ptr(A), A.shape[0], _ptr(B), B.shape[0], D, _ptr(dirs), nd, ka, kb,
                                   _ptr(idxA), ctypes.c_void_p(ns.data_ptr()), _ptr(idxB),
                                   ctypes.c_void_p(ns.data_ptr() + 8), _ptr(ws), ws.numel(), self._stream(stream))
        self._raise(rc, "prohd_select")
        return idxA, ns[0:1], idxB, ns[1:2]

    def prohd_estimate(self, A, B, params: Params | None = None, out=None, idxA=None, idxB=None, dirs=None,
                       ws=None, stream=None, **kw):
        """Enqueues prohd_estimate; returns the device result buffer (uint8 tensor)."""
        torch = _torch()
        _check_points(A, "A")
        _check_points(B, "B")
        p = params if params is not None else default_params(**kw)
        D = A.shape[1]
        need = self.lib.prohd_estimate_workspace_size(A.shape[0], B.shape[0], D, ctypes.byref(p))
        ws = self.workspace(need) if ws is None else ws
        out = torch.empty(ctypes.sizeof(Result), dtype=torch.uint8, device=A.device) if out is None else out
        rc = self.lib.prohd_estimate(self.h, _ptr(A), A.shape[0], _ptr(B), B.shape[0], D, ctypes.byref(p), _ptr(out),
                                     _ptr(idxA) if idxA is not None else None,
                                     _ptr(idxB) if idxB is not None else None,
                                     _ptr(dirs) if dirs is not None else None, _ptr(ws), ws.numel(),
                                     self._stream(stream))
        self._raise(rc, "prohd_estimate")
        return out

    def prohd_estimate_dirs(self, A, B, dirs, kA, kB, params: Params | None = None, out=None, idxA=None, idxB=None,
                            stream=None, **kw):
        """Enqueues prohd_estimate_dirs (selection onwards with the given
        directions dirs [nd, D] FP64 and k lists); returns the result buffer."""
        torch = _torch()
        _check_points(A, "A")
        _check_points(B, "B")
        p = params if params is not None else default_params(**kw)
        D = A.shape[1]
        dirs = dirs.to(device=A.device, dtype=torch.float64).contiguous()
        nd = dirs.shape[0]
        ka = (ctypes.c_int64 * nd)(*[int(k) for k in kA])
        kb = (ctypes.c_int64 * nd)(*[int(k) for k in kB])
        need = self.lib.prohd_estimate_dirs_workspace_size(A.shape[0], B.shape[0], D, nd, ka, kb, ctypes.byref(p))
        ws = self.workspace(need)
        out = torch.empty(ctypes.sizeof(Result), dtype=torch.uint8, device=A.device) if out is None else out
        rc = self.lib.prohd_estimate_dirs(self.h, _ptr(A), A.shape[0], _ptr(B), B.shape[0], D, ctypes.byref(p),
                                          _ptr(dirs), nd, ka, kb, _ptr(out),
                                          _ptr(idxA) if idxA is not None else None,
                                          _ptr(idxB) if idxB is not None else None, _ptr(ws), ws.numel(),
                                          self._stream(stream))
        self._raise(rc, "prohd_estimate_dirs")
        return out

    def prohd_estimate_adaptive(self, A, B, alpha_max, rel_tol, params: Params | None = None, out=None, idxA=None,
                                idxB=None, dirs=None, stream=None, **kw):
        """Runs the adaptive alpha schedule (synchronises the stream once per
        step); returns (device result buffer, decoded schedule dict)."""
        torch = _torch()
        _check_points(A, "A")
        _check_points(B, "B")
        p = params if params is not None else default_params(**kw)
        D = A.shape[1]
        need = self.lib.prohd_estimate_adaptive_workspace_size(A.shape[0], B.shape[0], D, ctypes.byref(p),
                                                              float(alpha_max))
        ws = self.workspace(need)
        out = torch.empty(ctypes.sizeof(Result), dtype=torch.uint8, device=A.device) if out is None else out
        info = AdaptiveInfo()
        rc = self.lib.prohd_estimate_adaptive(self.h, _ptr(A), A.shape[0], _ptr(B), B.shape[0], D, ctypes.byref(p),
                                              float(alpha_max), float(rel_tol), _ptr(out), ctypes.byref(info),
                                              _ptr(idxA) if idxA is not None else None,
                                              _ptr(idxB) if idxB is not None else None,
                                              _ptr(dirs) if dirs is not None else None, _ptr(ws), ws.numel(),
                                              self._stream(stream))
        self._raise(rc, "prohd_estimate_adaptive")
        n = info.steps
        sched = dict(steps=n, reason=ADAPT_REASONS.get(info.reason, info.reason), alpha_c=info.alpha_c,
                     alpha_p=info.alpha_p, H=list(info.H[:n]), nsel_a=list(info.nsel_a[:n]),
                     nsel_b=list(info.nsel_b[:n]))
        return out, sched

    def prohd_features(self, A, B, feat=None, dirs=None, eig=None, seed=0, stream=None):
        """Network input features [10 D] (FP32), directions [9, D] and eig [8] of a pair."""
        torch = _torch()
        _check_points(A, "A")
        _check_points(B, "B")
        D = A.shape[1]
        p = default_params(m=8, seed=seed)
        feat = torch.empty(10 * D, dtype=torch.float32, device=A.device) if feat is None else feat
        dirs = torch.empty((9, D), dtype=torch.float64, device=A.device) if dirs is None else dirs
        eig = torch.empty(8, dtype=torch.float64, device=A.device) if eig is None else eig
        ws = self.workspace(self.lib.prohd_features_workspace_size(A.shape[0], B.shape[0], D))
        rc = self.lib.prohd_features(self.h, _ptr(A), A.shape[0], _ptr(B), B.shape[0], D, ctypes.byref(p), _ptr(feat),
                                     _ptr(dirs), _ptr(eig), _ptr(ws), ws.numel(), self._stream(stream))
        self._raise(rc, "prohd_features")
        return feat, dirs, eig

    def prohd_estimate_host(self, A_host, B_host, params: Params | None = None, out_host=None, ws=None,
                            stream=None, **kw):
        """A_host, B_host: CPU float32 tensors (pinned for async copies). Returns
        the host Result that is valid after the stream is synchronised."""
        torch = _torch()
        for t, nme in ((A_host, "A_host"), (B_host, "B_host")):
            if t.device.type != "cpu" or t.dtype != torch.float32 or t.dim() != 2 or not t.is_contiguous():
                raise ValueError(f"{nme} must be a contiguous CPU float32 tensor [n, D]")
        p = params if params is not None else default_params(**kw)
        D = A_host.shape[1]
        need = self.lib.prohd_estimate_host_workspace_size(A_host.shape[0], B_host.shape[0], D, ctypes.byref(p))
        ws = self.workspace(need) if ws is None else ws
        out_host = Result() if out_host is None else out_host
        rc = self.lib.prohd_estimate_host(self.h, _ptr(A_host), A_host.shape[0], _ptr(B_host), B_host.shape[0], D,
                                          ctypes.byref(p), ctypes.byref(out_host), _ptr(ws), ws.numel(),
                                          self._stream(stream))
        self._raise(rc, "prohd_estimate_host")
        return out_host


class Batch:
    """A planned batch of independent pairs (prohd_batch_plan). Keeps the
    pair tensors and the workspace alive for the plan's lifetime."""

    def __init__(self, ctx: Context, pairs, params: Params | None = None, **kw):
        torch = _torch()
        self.ctx = ctx
        self.params = params if params is not None else default_params(**kw)
        self.pairs = []
        for A, B in pairs:
            _check_points(A, "A")
            _check_points(B, "B")
            if A.shape[1] != B.shape[1]:
                raise ValueError("A and B of a pair must have the same D")
            self.pairs.append((A, B))
        n = len(self.pairs)
        self._desc = (PairDesc * n)()
        for i, (A, B) in enumerate(self.pairs):
            self._desc[i] = PairDesc(A.data_ptr(), A.shape[0], B.data_ptr(), B.shape[0], A.shape[1], 0)
        need = ctx.lib.prohd_batch_workspace_size(self._desc, n, ctypes.byref(self.params))
        if need == 0:
            # let the planner report why
            need = 256
        dev = self.pairs[0][0].device
        self.ws = torch.empty(int(need), dtype=torch.uint8, device=dev)
        self.out = torch.empty(n * ctypes.sizeof(Result), dtype=torch.uint8, device=dev)
        h = ctypes.c_void_p()
        rc = ctx.lib.prohd_batch_plan(ctx.h, self._desc, n, ctypes.byref(self.params), _ptr(self.ws), self.ws.numel(),
                                      ctypes.byref(h))
        ctx._raise(rc, "prohd_batch_plan")
        self.h = h
        self.n = n

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.prohd_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def use_graph(self, on: bool):
        self.ctx._raise(self.ctx.lib.prohd_batch_use_graph(self.h, 1 if on else 0), "prohd_batch_use_graph")

    def run(self, stream=None):
        """Enqueues the whole batch; returns the device result buffer."""
        rc = self.ctx.lib.prohd_estimate_batched(self.ctx.h, self.h, _ptr(self.out), self.ctx._stream(stream))
        self.ctx._raise(rc, "prohd_estimate_batched")
        return self.out

    def autotune(self, stream=None) -> float:
        ms = ctypes.c_double()
        rc = self.ctx.lib.prohd_batch_autotune(self.ctx.h, self.h, _ptr(self.out), self.ctx._stream(stream),
                                               ctypes.byref(ms))
        self.ctx._raise(rc, "prohd_batch_autotune")
        return ms.value

    def tunables(self) -> dict:
        g, p, s = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self.ctx._raise(self.ctx.lib.prohd_batch_get_tunables(self.h, ctypes.byref(g), ctypes.byref(p),
                                                              ctypes.byref(s)), "prohd_batch_get_tunables")
        return dict(gram_pts=g.value, proj_rows=p.value, sel_chunk=s.value)

    def set_tunables(self, gram_pts: int, proj_rows: int, sel_chunk: int):
        self.ctx._raise(self.ctx.lib.prohd_batch_set_tunables(self.h, gram_pts, proj_rows, sel_chunk),
                        "prohd_batch_set_tunables")

    def results(self) -> list:
        """Decodes the result buffer (call after the stream is synchronised)."""
        host = bytes(self.out.cpu().numpy().tobytes())
        sz = ctypes.sizeof(Result)
        return [decode_result(Result.from_buffer_copy(host[i * sz:(i + 1) * sz])) for i in range(self.n)]

    def iterations(self) -> np.ndarray:
        """Block-iteration steps of every pair in the last run (after a synchronise)."""
        torch = _torch()
        out = np.zeros(self.n, dtype=np.int64)
        base = self.ws.data_ptr()
        for i in range(self.n):
            it = ctypes.c_void_p()
            self.ctx._raise(self.ctx.lib.prohd_batch_pair_outputs(self.h, i, None, None, None, ctypes.byref(it)),
                            "prohd_batch_pair_outputs")
            off = it.value - base
            out[i] = int(self.ws[off:off + 4].view(torch.int32).item())
        return out

    def pair_outputs(self, i: int, nsel_a: int, nsel_b: int):
        """(dirs [1+m, D] float64, idxA [nsel_a], idxB [nsel_b]) of pair i as numpy arrays."""
        torch = _torch()
        d, a, b = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        self.ctx._raise(self.ctx.lib.prohd_batch_pair_outputs(self.h, i, ctypes.byref(d), ctypes.byref(a),
                                                              ctypes.byref(b), None), "prohd_batch_pair_outputs")
        A, _ = self.pairs[i]
        D = A.shape[1]
        m = self.params.m if self.params.m >= 0 else int(math.isqrt(D))
        base = self.ws.data_ptr()

        def view(ptr, count, dtype, itemsize):
            off = ptr - base
            return self.ws[off:off + count * itemsize].view(dtype)

        dirs = view(d.value, (1 + m) * D, torch.float64, 8).reshape(1 + m, D).cpu().numpy()
        ia = view(a.value, nsel_a, torch.int32, 4).cpu().numpy().astype(np.int64)
        ib = view(b.value, nsel_b, torch.int32, 4).cpu().numpy().astype(np.int64)
        return dirs, ia, ib


class Mlp:
    """The learned-direction network: FP32 state (params | Adam m | Adam v)
    and a scratch buffer on the device; every computation runs in the
    library's kernels."""

    MAGIC = b"PHDMLP01"

    def __init__(self, ctx: Context, D: int, seed: int = 0, device=None, init: bool = True):
        torch = _torch()
        self.ctx, self.D = ctx, int(D)
        dev = device if device is not None else f"cuda:{ctx.device}"
        self.nparam = int(ctx.lib.prohd_mlp_param_count(self.D))
        self.state = torch.zeros(3 * self.nparam, dtype=torch.float32, device=dev)
        self.step = 0
        self._scratch = None
        self._batch = 0
        if init:
            self.init(seed)

    def init(self, seed: int, stream=None):
        rc = self.ctx.lib.prohd_mlp_init(self.ctx.h, self.D, int(seed), _ptr(self.state), self.ctx._stream(stream))
        self.ctx._raise(rc, "prohd_mlp_init")
        self.step = 0

    def scratch(self, batch: int):
        torch = _torch()
        need = int(self.ctx.lib.prohd_mlp_scratch_bytes(self.D, batch))
        if self._scratch is None or self._scratch.numel() < need:
            self._scratch = torch.empty(need, dtype=torch.uint8, device=self.state.device)
        return self._scratch

    @property
    def params(self):
        return self.state[: self.nparam]

    def forward(self, feat, precision="bf16", want64=False, stream=None):
        """Unit directions [B, 4, D] (FP32), and FP64 [B, 4, D] when want64."""
        torch = _torch()
        feat = feat.reshape(-1, 10 * self.D).contiguous()
        B = feat.shape[0]
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        u = torch.empty((B, 4, self.D), dtype=torch.float32, device=feat.device)
        u64 = torch.empty((B, 4, self.D), dtype=torch.float64, device=feat.device) if want64 else None
        sc = self.scratch(B)
        rc = self.ctx.lib.prohd_mlp_forward(self.ctx.h, self.D, _ptr(self.state), _ptr(feat), B, prec, _ptr(u),
                                            _ptr(u64) if want64 else None, _ptr(sc), sc.numel(),
                                            self.ctx._stream(stream))
        self.ctx._raise(rc, "prohd_mlp_forward")
        return (u, u64) if want64 else u

    def loss_grad(self, feat, label, precision="fp32", want_grad=True, stream=None):
        torch = _torch()
        feat = feat.reshape(-1, 10 * self.D).contiguous()
        label = label.reshape(-1, self.D).contiguous()
        B = feat.shape[0]
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        loss = torch.empty(1, dtype=torch.float32, device=feat.device)
        grad = torch.empty(self.nparam, dtype=torch.float32, device=feat.device) if want_grad else None
        sc = self.scratch(B)
        rc = self.ctx.lib.prohd_mlp_loss_grad(self.ctx.h, self.D, _ptr(self.state), _ptr(feat), _ptr(label), B, prec,
                                              _ptr(loss), _ptr(grad) if want_grad else None, _ptr(sc), sc.numel(),
                                              self.ctx._stream(stream))
        self.ctx._raise(rc, "prohd_mlp_loss_grad")
        return loss, grad

    def train_step(self, feat, label, lr=1e-3, precision="bf16", loss=None, stream=None):
        """One Adam step; returns the device loss (mean over the batch, before the step)."""
        torch = _torch()
        B = feat.shape[0]
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        loss = torch.empty(1, dtype=torch.float32, device=feat.device) if loss is None else loss
        sc = self.scratch(B)
        self.step += 1
        rc = self.ctx.lib.prohd_mlp_train_step(self.ctx.h, self.D, _ptr(self.state), _ptr(feat), _ptr(label), B, prec,
                                               ctypes.c_float(lr), self.step, _ptr(loss), _ptr(sc), sc.numel(),
                                               self.ctx._stream(stream))
        self.ctx._raise(rc, "prohd_mlp_train_step")
        return loss

    def adam(self, grad, lr=1e-3, stream=None):
        """One Adam step with a given gradient [param_count] (device FP32)."""
        self.step += 1
        rc = self.ctx.lib.prohd_mlp_adam_step(self.ctx.h, self.D, _ptr(self.state), _ptr(grad.contiguous()),
                                              ctypes.c_float(lr), self.step, self.ctx._stream(stream))
        self.ctx._raise(rc, "prohd_mlp_adam_step")

    # ------------------------------------------------------------- checkpoints

    def save(self, path: str, rng_state: bytes = b"", stream=None):
        """Versioned checkpoint through prohd_mlp_save: magic, D, step,
        parameter count, the host RNG state of the training sampler, then
        params, Adam m, Adam v."""
        buf = ctypes.create_string_buffer(rng_state, len(rng_state)) if rng_state else None
        rc = self.ctx.lib.prohd_mlp_save(self.ctx.h, os.fsencode(path), self.D, self.step, _ptr(self.state),
                                         buf, len(rng_state), self.ctx._stream(stream))
        self.ctx._raise(rc, "prohd_mlp_save")

    @classmethod
    def load(cls, ctx: Context, path: str, device=None, stream=None):
        """Returns (network, rng_state), through prohd_mlp_load."""
        D, step, nx = ctypes.c_int32(0), ctypes.c_int64(0), ctypes.c_int64(0)
        rc = ctx.lib.prohd_mlp_load(ctx.h, os.fsencode(path), ctypes.byref(D), ctypes.byref(step), None, None, 0,
                                    ctypes.byref(nx), ctx._stream(stream))
        if rc != PROHD_OK:
            raise ValueError(f"{path}: {ctx.lib.prohd_last_error(ctx.h).decode()}")
        net = cls(ctx, D.value, init=False, device=device)
        buf = ctypes.create_string_buffer(max(nx.value, 1))
        rc = ctx.lib.prohd_mlp_load(ctx.h, os.fsencode(path), ctypes.byref(D), ctypes.byref(step), _ptr(net.state),
                                    buf, nx.value, ctypes.byref(nx), ctx._stream(stream))
        if rc != PROHD_OK:
            raise ValueError(f"{path}: {ctx.lib.prohd_last_error(ctx.h).decode()}")
        net.step = step.value
        return net, buf.raw[: nx.value]


# ----------------------------------------------------------------- decoding

def _decode(buf, cls):
    host = bytes(buf.cpu().numpy().tobytes()) if hasattr(buf, "cpu") else bytes(buf)
    return cls.from_buffer_copy(host)


def hd_dict(r: HdResult) -> dict:
    return dict(H=r.H, h_ab=r.h_ab, h_ba=r.h_ba, wit_a=r.wit_a, wit_b=r.wit_b, ab=(r.ab_a, r.ab_b),
                ba=(r.ba_b, r.ba_a), dir=r.dir, status=STATUS_NAMES.get(r.status, r.status), H_lowp=r.H_lowp,
                n_rescored_a=r.n_rescored_a, n_rescored_b=r.n_rescored_b)


def decode_hd(buf) -> dict:
    return hd_dict(_decode(buf, HdResult))


def decode_result(buf) -> dict:
    r = _decode(buf, Result) if not isinstance(buf, Result) else buf
    d = hd_dict(r.hd)
    d.update(nsel_a=r.nsel_a, nsel_b=r.nsel_b)
    return d


_default_ctx = None


def context() -> Context:
    global _default_ctx
    if _default_ctx is None:
        _default_ctx = Context()
    return _default_ctx


def hausdorff_exact_sync(A, B, precision="fp16") -> dict:
    torch = _torch()
    out = context().hausdorff_exact(A, B, precision)
    torch.cuda.current_stream().synchronize()
    return decode_hd(out)


def prohd_estimate_sync(A, B, want_indices=False, want_dirs=False, **kw) -> dict:
    torch = _torch()
    ctx = context()
    idxA = torch.empty(A.shape[0], dtype=torch.int32, device=A.device) if want_indices else None
    idxB = torch.empty(B.shape[0], dtype=torch.int32, device=A.device) if want_indices else None
    dirs = None
    if want_dirs:
        D = A.shape[1]
        m = kw.get("m")
        m = int(math.isqrt(D)) if m is None or m < 0 else int(m)
        dirs = torch.empty((1 + m, D), dtype=torch.float64, device=A.device)
    out = ctx.prohd_estimate(A, B, idxA=idxA, idxB=idxB, dirs=dirs, **kw)
    torch.cuda.current_stream().synchronize()
    r = decode_result(out)
    if want_dirs:
        r["dirs"] = dirs.cpu().numpy()
    if want_indices:
        r["idxA"] = idxA[: r["nsel_a"]].cpu().numpy().astype(np.int64)
        r["idxB"] = idxB[: r["nsel_b"]].cpu().numpy().astype(np.int64)
    return r
