"""The C-ABI library builds and loads, and exports every function that
include/gr.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(gr_[a-z0-9_]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libgr():
    import shutil
    from paper_2303_15762_gb300 import build
    if not os.path.exists(build.LIB):
        if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
            pytest.skip("nvcc not available to build libgr.so")
        build.build()
    return ctypes.CDLL(build.LIB)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["gr_scene_create", "gr_scene_destroy", "gr_render", "gr_readback", "gr_frame_create",
                     "gr_frame_release", "gr_last_error"]:
        assert required in names, names


def test_library_exports_every_declared_symbol(libgr):
    for name in _declared_functions():
        assert hasattr(libgr, name), name


def test_binding_lists_match_header():
    from paper_2303_15762_gb300 import _native
    assert set(_native.EXPORTED) <= set(_declared_functions())


def test_abi_version_and_error_string_without_gpu(libgr):
    libgr.gr_abi_version.restype = ctypes.c_int32
    assert libgr.gr_abi_version() == 1
    libgr.gr_last_error.restype = ctypes.c_char_p
    assert isinstance(libgr.gr_last_error(), bytes)


def test_null_arguments_rejected_without_gpu(libgr):
    """Argument validation happens before any CUDA call."""
    libgr.gr_scene_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert libgr.gr_scene_create(None, None, None) == 1
    libgr.gr_render.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                ctypes.c_void_p, ctypes.c_void_p]
    assert libgr.gr_render(None, 0, None, 0, None, None, None) == 1
