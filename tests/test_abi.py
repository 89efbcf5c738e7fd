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


def test_binding_covers_the_header_exactly():
    # the binding declares a ctypes signature for every C entry point and for nothing else
    import paper_2109_05072_gb300 as ceed
    assert set(ceed._SIGNATURES) == set(_declared())


def test_binding_refuses_host_tensors():
    # device arguments must be CUDA tensors: there is no CPU path to fall back to
    torch = __import__("pytest").importorskip("torch")
    import pytest
    import paper_2109_05072_gb300 as ceed
    with pytest.raises(ValueError):
        ceed._ptr(torch.zeros(4, dtype=torch.float64))
    with pytest.raises(ValueError):          # host buffers of ceed_apply_host must be FP64
        ceed._host_ptr(torch.zeros(4, dtype=torch.float32))
    assert ceed._host_ptr(torch.zeros(4, dtype=torch.float64)).value != 0


def test_import_fails_loudly_without_the_library():
    import subprocess
    import sys
    # the build module is loaded on its own and registered first, so that the package's
    # `from .build import LIB` sees the missing path
    code = ("import importlib.util, os, sys; sys.path.insert(0, %r)\n"
            "spec = importlib.util.spec_from_file_location('paper_2109_05072_gb300.build',\n"
            "    os.path.join(sys.path[0], 'paper_2109_05072_gb300', 'build.py'))\n"
            "b = importlib.util.module_from_spec(spec); spec.loader.exec_module(b)\n"
            "b.LIB = '/nonexistent/libceedgb.so'\n"
            "sys.modules['paper_2109_05072_gb300.build'] = b\n"
            "try:\n"
            "    import paper_2109_05072_gb300\n"
            "except ImportError as e:\n"
            "    print('refused:', e)\n"
            "else:\n"
            "    print('imported')\n") % ROOT
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    assert "refused:" in r.stdout and "not built" in r.stdout, r.stdout + r.stderr


def test_struct_layouts_match_header(tmp_path):
    # every ctypes mirror of a header struct has the C layout: gcc compiles a probe against the
    # header that prints sizeof and each field's offset, compared with ctypes' own
    import ctypes
    import shutil
    import subprocess
    import pytest
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    import paper_2109_05072_gb300 as ceed
    mirrors = {"ceed_mesh_desc": ceed._MeshDesc, "ceed_cg_opts": ceed._CgOpts, "ceed_cg_report": ceed._CgReport,
               "ceed_pmg_opts": ceed._PmgOpts, "ceed_nt_desc": ceed._NtDesc, "ceed_hp_desc": ceed._HpDesc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ceed_gb300.h"', "int main(void) {"]
    for cname, cls in mirrors.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True, timeout=120)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.split("\n")
    got = {}
    for line in out:
        if line.strip():
            cname, field, value = line.split()
            got[(cname, field)] = int(value)
    for cname, cls in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_wait_limits_validated_on_the_host():
    # limits above the defaults are refused before anything reaches a device; -1 restores them
    import paper_2109_05072_gb300 as ceed
    assert ceed._lib.ceed_set_wait_limits(1 << 23, -1) == ceed.CEED_ERR_INVALID
    assert ceed._lib.ceed_set_wait_limits(5, -1) == ceed.CEED_ERR_INVALID
    assert ceed._lib.ceed_set_wait_limits(-1, 1 << 26) == ceed.CEED_ERR_INVALID
    assert ceed._lib.ceed_set_wait_limits(-1, -1) == ceed.CEED_OK
    assert ceed._lib.ceed_fma_throughput(5, None, None, None, None) == ceed.CEED_ERR_INVALID
    assert ceed._lib.ceed_fma_throughput(-1, None, None, None, None) == ceed.CEED_ERR_INVALID
