"""Host-side checks of the C ABI: the library builds, loads without a GPU, exports every symbol
include/rs.h declares, the binding declares the same set, and calls fail cleanly without a device."""

import ctypes
import os
import re

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rs.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rs_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def librs():
    from paper_1602_02350_gb300 import _lib, build
    build.build()          # incremental: recompiles only sources newer than their objects
    return _lib.lib()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("rs_sketch", "rs_precondition", "rs_svrg_solve", "rs_full_gradient", "rs_svrg_epoch",
                     "rs_index_stream", "rs_countsketch", "rs_objective", "rs_solve"):
        assert required in names


def test_library_exports_every_declared_symbol(librs):
    missing = [n for n in _declared() if not hasattr(librs, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_1602_02350_gb300 import _lib
    assert sorted(_lib.declared_symbols()) == _declared()
    import paper_1602_02350_gb300 as pkg
    for n in _declared():
        if n not in ("rs_create", "rs_destroy", "rs_set_stream", "rs_last_error", "rs_abi_version",
                     "rs_launch_count"):
            assert hasattr(pkg, n), n


def test_abi_version(librs):
    assert librs.rs_abi_version() == 1


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device path")
def test_no_device_fails_cleanly(librs):
    h = ctypes.c_void_p()
    rc = librs.rs_create(ctypes.byref(h), 0, None)
    assert rc == 3                       # RS_ECUDA
    assert b"no CUDA device" in librs.rs_last_error()
    assert librs.rs_launch_count(None) == -1
    # null context is rejected before any CUDA call
    assert librs.rs_philox_words(None, 0, 0, 0, 4, None) == 1


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device path")
def test_python_binding_refuses_without_gpu():
    from paper_1602_02350_gb300 import Context
    with pytest.raises(RuntimeError):
        Context(0)
