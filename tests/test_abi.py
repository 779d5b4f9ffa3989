"""The C-ABI library builds, loads without a GPU, and exports every entry
point that include/prohd.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_2511_18207_gb300 import build_lib, prohd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "prohd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n.startswith(("prohd_", "hausdorff_"))))


def test_header_lists_the_binding_exports():
    assert _declared() == sorted(prohd.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = build_lib.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_host_only_helpers():
    prohd.load_library()
    assert prohd.k_of(0.01, 2000) == 20
    assert prohd.k_of(0.5, 1) == 1
    p = prohd.default_params()
    assert p.m == -1 and p.precision == 1 and p.alpha_c == 0.01 and p.power_max_iters == 96


def test_batch_workspace_size_is_host_only():
    # planning checks run on the host: valid pairs get a size, invalid ones 0
    lib = prohd.load_library()
    p = prohd.default_params(m=8)
    ok = (prohd.PairDesc * 2)(prohd.PairDesc(256, 1000, 512, 2000, 64, 0),
                              prohd.PairDesc(1024, 5000, 2048, 300, 256, 0))
    n = lib.prohd_batch_workspace_size(ok, 2, ctypes.byref(p))
    assert n > 0
    big = (prohd.PairDesc * 1)(prohd.PairDesc(256, 100_000, 512, 100_000, 256, 0))
    assert lib.prohd_batch_workspace_size(big, 1, ctypes.byref(p)) > n
    for D, a in ((13, 256), (512, 256), (64, 4)):
        bad = (prohd.PairDesc * 1)(prohd.PairDesc(a, 1000, 512, 2000, D, 0))
        assert lib.prohd_batch_workspace_size(bad, 1, ctypes.byref(p)) == 0, (D, a)
    p30 = prohd.default_params(m=30)
    assert lib.prohd_batch_workspace_size(ok, 2, ctypes.byref(p30)) == 0
    # the one-sided refinement adds, per pair, rounded copies of both whole
    # sets (tensor precisions) or the FP32 path's minima: more room, and more
    # with the larger sets; refine must be 0 or 1
    for prec in (1, 2, 0):
        p0 = prohd.default_params(m=8, precision=prec)
        p1 = prohd.default_params(m=8, precision=prec, refine=1)
        n0 = lib.prohd_batch_workspace_size(ok, 2, ctypes.byref(p0))
        n1 = lib.prohd_batch_workspace_size(ok, 2, ctypes.byref(p1))
        assert n1 > n0 > 0, (prec, n0, n1)
    p1 = prohd.default_params(m=8, refine=1)
    n_small = lib.prohd_batch_workspace_size(ok, 2, ctypes.byref(p1)) - n
    n_big = lib.prohd_batch_workspace_size(big, 1, ctypes.byref(p1)) - \
        lib.prohd_batch_workspace_size(big, 1, ctypes.byref(p))
    assert n_big > n_small > 0
    p2 = prohd.default_params(m=8, refine=2)
    assert lib.prohd_batch_workspace_size(ok, 2, ctypes.byref(p2)) == 0


def test_new_entry_points_size_their_workspaces_on_the_host():
    lib = prohd.load_library()
    # pruned exact distance: the plain size below 32,768 rows or with FP32
    for nA, nB, prec in ((1000, 2000, 1), (100_000, 90_000, 0)):
        assert lib.hausdorff_exact_pruned_workspace_size(nA, nB, 64, prec) == \
            lib.hausdorff_exact_workspace_size(nA, nB, 64, prec)
    assert lib.hausdorff_exact_pruned_workspace_size(100_000, 90_000, 64, 1) > 0
    # the refinement needs more room than the plain estimate
    p0 = prohd.default_params(m=4)
    p1 = prohd.default_params(m=4, refine=1)
    assert lib.prohd_estimate_workspace_size(50_000, 40_000, 64, ctypes.byref(p1)) > \
        lib.prohd_estimate_workspace_size(50_000, 40_000, 64, ctypes.byref(p0))
    # adaptive alpha: sized for the largest step the budget allows; 0 when
    # the budget is below the first step
    small = lib.prohd_estimate_adaptive_workspace_size(50_000, 40_000, 64, ctypes.byref(p0), 0.01)
    large = lib.prohd_estimate_adaptive_workspace_size(50_000, 40_000, 64, ctypes.byref(p0), 0.3)
    assert 0 < small < large
    assert lib.prohd_estimate_adaptive_workspace_size(50_000, 40_000, 64, ctypes.byref(p0), 0.005) == 0
