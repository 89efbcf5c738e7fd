"""The C-ABI library loads on a machine without a GPU and exports every entry point the header declares."""
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ceed_gb300.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ceed_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def _build_module():
    spec = importlib.util.spec_from_file_location("_ceedgb_build", os.path.join(ROOT, "paper_2109_05072_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_header_symbols_exported():
    lib_path = _build_module().build()
    import ctypes
    lib = ctypes.CDLL(lib_path)
    names = _declared()
    for core in ("ceed_setup_mesh", "ceed_build_qdata", "ceed_apply_mass", "ceed_apply_diffusion", "ceed_cg_solve"):
        assert core in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding wraps every declared entry point under the same name
    import paper_2109_05072_gb300 as ceed
    assert set(names) <= set(ceed.EXPORTED)
    for n in names:
        assert callable(getattr(ceed, n)), n


def test_last_error_without_gpu():
    import paper_2109_05072_gb300 as ceed
    # a call that fails on argument validation touches no device
    assert ceed._lib.ceed_setup_mesh(None, None, None) == ceed.CEED_ERR_INVALID
    assert "null" in ceed.ceed_last_error()
    assert ceed.ceed_dot_noalloc_max_n() == 32768 * 8192
