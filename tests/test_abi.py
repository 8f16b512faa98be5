"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every entry point include/mpkm.h declares.  No compute call (no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mpkm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(km_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2407_12208_gb300 import build
    lib = build.build()
    names = _declared()
    assert "km_assign" in names and "km_submit" in names
    so = ctypes.CDLL(lib)
    for n in names:
        assert hasattr(so, n), n
    import paper_2407_12208_gb300 as pkg
    assert sorted(pkg.EXPORTS) == names


def test_binding_refuses_without_library(tmp_path):
    from paper_2407_12208_gb300 import _binding
    with pytest.raises(RuntimeError):
        _binding._lib = None
        _binding.load(str(tmp_path / "missing.so"))
    _binding._lib = None


def test_default_params_and_workspace_query():
    import paper_2407_12208_gb300 as pkg
    pkg.load()
    p = pkg.params()
    assert p.low == pkg.BF16 and p.test == pkg.TEST_TC and p.rho == 5.0 and p.paper_factor == 2.0
    lib = pkg.load()
    # km_workspace_size with a NULL context is rejected, not a crash
    b = ctypes.c_size_t()
    assert lib.km_workspace_size(None, 10, 4, 2, ctypes.byref(p), ctypes.byref(b)) == 1
