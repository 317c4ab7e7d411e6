"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/*.h declares (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:cg_status|const char\*|void)\s+(cg_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib_path():
    from paper_1604_06667_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_symbols()
    for n in ("cg_grid_create", "cg_set_kernel", "cg_grid_add", "cg_grid_finalize",
              "cg_grid_destroy", "cg_last_error", "cg_ang2pix_ring"):
        assert n in names


def test_library_loads_and_exports_everything(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol(lib_path):
    from paper_1604_06667_gb300 import _capi
    lib = _capi.load(lib_path)
    for n in declared_symbols():
        if n == "cg_last_error":
            continue
        assert n in _capi.SIGNATURES, n
        assert hasattr(_capi, n), n
    assert lib.cg_last_error() == b""


def test_only_the_c_abi_is_exported(lib_path):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    assert exported == declared_symbols(), exported ^ declared_symbols()


def test_argument_errors_without_gpu(lib_path):
    """Host-side argument checks return CG_EINVAL before touching the device."""
    from paper_1604_06667_gb300 import _capi
    lib = _capi.load(lib_path)
    h = ctypes.c_void_p()
    assert lib.cg_grid_create(ctypes.byref(h), None, None, 10, 1, None) == _capi.CG_EINVAL
    assert b"null" in lib.cg_last_error()
    assert lib.cg_grid_create(None, None, None, 10, 1, None) == _capi.CG_EINVAL
    assert lib.cg_ang2pix_ring(0, None, None, 1, None, None) == _capi.CG_EINVAL
    assert lib.cg_set_kernel(None, 0, None, 0, 1.0, 0, 1.0) == _capi.CG_EINVAL
    assert lib.cg_grid_add(None, None, None, None, 0, None, 1) == _capi.CG_EINVAL
