"""The C ABI library builds, loads without a GPU, and exports every entry
point that include/*.h declares (no compute call is made here)."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"^[A-Za-z_][\w \*]*?\b(fp_\w+)\s*\(", txt, flags=re.M))
    return names


def test_header_declares_the_four_calls():
    names = _declared()
    assert "fp_closure_exact" in names and "fp_workspace_bytes" in names


def test_library_exports_every_declared_symbol():
    from paper_2606_15622_gb300 import api
    L = ctypes.CDLL(api.library_path()) if os.path.exists(api.library_path()) else api.lib()
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2606_15622_gb300 import api
    assert _declared() <= set(api.SIGNATURES)


def test_host_only_calls_work_without_gpu():
    from paper_2606_15622_gb300 import api
    L = api.lib()
    assert L.fp_version() >= 100
    assert L.fp_status_string(-1) == b"invalid argument"
    p = api.default_params()
    assert p.min_particles == 4 and p.pivot_rtol == 1e-13
    assert api.workspace_bytes(1000, 5000, "fp32") == 256 * ((1000 * 30 * 8 + 255) // 256)
    assert api.workspace_bytes(1000, 5000, "fp32", moments_out_given=True) == 0
