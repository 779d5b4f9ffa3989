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
    assert p.m == -1 and p.precision == 1 and p.alpha_c == 0.01 and p.power_max_iters == 1000
