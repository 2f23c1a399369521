"""The C-ABI library builds for sm_103a, loads, and exports every function include/hwswe.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "hwswe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hw_[a-z0-9_]+)\s*\(", src)))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_exports_every_declared_symbol():
    from paper_2208_01260_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared()
    assert "hw_create" in names and "hw_rk3_step" in names and "hw_advance" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    lib.hw_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.hw_version()


def test_argument_checks_without_gpu():
    """Argument validation happens before any CUDA call."""
    import paper_2208_01260_gb300 as hw
    try:
        hw.lib()
    except RuntimeError:
        pytest.skip("library not built")
    out = ctypes.c_void_p()
    g = hw.make_grid(1, 1, dim=2)
    rc = hw.lib().hw_create(ctypes.byref(g), ctypes.byref(hw.make_params()), None, ctypes.byref(out))
    assert rc == -1 and b"nx" in hw.lib().hw_last_error()
    assert hw.lib().hw_rk3_step(None, 1.0) == -1
