"""The C-ABI library builds, loads without a GPU, and exports every function include/klst.h declares."""
import ctypes
import os
import re

from paper_2607_27440_b300 import build, klst

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "klst.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(klst_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("klst_build_pencil", "klst_factor_shift", "klst_apply_shift_invert", "klst_eigs"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.LIB)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(klst.EXPORTS) | {"klst_stream"}


def test_status_strings_without_gpu():
    lib = klst.load()
    assert lib.klst_status_string(-3) == b"KLST_ESINGULAR"
    assert lib.klst_status_string(0) == b"KLST_OK"


def test_invalid_descriptor_rejected_before_device_work():
    lib = klst.load()
    d = klst.PencilDesc(nx=2, qx=4, qy=4, map_L=1, map_sinf=30, mach=2, gamma=5 / 3, visc_s=0.5, re_delta=10,
                        beta=1, width=0.5, base=1, noneq=1, conservative=1)
    h = ctypes.c_void_p()
    assert lib.klst_build_pencil(ctypes.byref(d), None, ctypes.byref(h)) == klst.KLST_EINVAL
    assert h.value is None
    assert b"unsupported sizes" in lib.klst_last_error()
