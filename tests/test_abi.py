"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/sgpe.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sgpe_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2009_13507_gb300 import build as B
    lib_path = B.build()
    lib = ctypes.CDLL(lib_path)
    names = _declared("sgpe.h")
    assert "sgpe_step_imag" in names and "sgpe_energy" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_every_declared_symbol():
    from paper_2009_13507_gb300 import sgpe
    assert sorted(sgpe.EXPORTS) == _declared("sgpe.h")


def test_init_rejects_bad_arguments_without_gpu():
    """Argument checks happen before any CUDA call."""
    from paper_2009_13507_gb300 import sgpe
    lib = sgpe.load()
    ctx = ctypes.c_void_p()
    assert lib.sgpe_init_grid(ctypes.byref(ctx), 3, 16, 16, 0.1, 0.1, 0, None) == sgpe.EINVAL
    assert lib.sgpe_init_grid(ctypes.byref(ctx), 2, 2, 16, 0.1, 0.1, 0, None) == sgpe.EINVAL
    assert lib.sgpe_init_grid(ctypes.byref(ctx), 2, 16, 16, -0.1, 0.1, 0, None) == sgpe.EINVAL
    assert lib.sgpe_init_grid(ctypes.byref(ctx), 2, 5000, 16, 0.1, 0.1, 0, None) == sgpe.EUNSUPPORTED
    assert lib.sgpe_init_grid(ctypes.byref(ctx), 2, 16, 16, 0.1, 0.1, 7, None) == sgpe.EINVAL
    assert lib.sgpe_init_grid(None, 2, 16, 16, 0.1, 0.1, 0, None) == sgpe.EINVAL
    assert lib.sgpe_destroy(None) == sgpe.OK
