"""Host-side checks of the C ABI: the library builds and loads, exports every
symbol include/adiwave.h declares, and rejects bad arguments before touching
a GPU.  No compute call is made here."""
import ctypes
import os
import re

import pytest

from paper_2006_10142_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(adi_wave_\w+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    return _lib.load()


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("adi_wave_init", "adi_wave_step", "adi_wave_run", "adi_wave_adjoint"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert names, "no declarations found"
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_lib.EXPORTS) == names


def test_strerror_and_version(lib):
    for code in range(8):
        assert lib.adi_wave_strerror(code)
    assert b"sm_103a" in lib.adi_wave_version()


def test_init_rejects_bad_arguments_without_gpu(lib):
    h = ctypes.c_void_p()
    one = (ctypes.c_void_p * 1)(1)
    bad_descs = [
        _lib.Desc(0, 10, 1.0, 1.0, 0.01, 0, 0),      # nx < 1
        _lib.Desc(10, 40000, 1.0, 1.0, 0.01, 0, 0),  # ny too large
        _lib.Desc(10, 10, 0.0, 1.0, 0.01, 0, 0),     # lx <= 0
        _lib.Desc(10, 10, 1.0, 1.0, -1.0, 0, 0),     # dt <= 0
        _lib.Desc(10, 10, 1.0, 1.0, 0.01, 5, 0),     # bad start mode
        _lib.Desc(10, 10, 1.0, 1.0, 0.01, 0, 9),     # bad fp64 mode
    ]
    for d in bad_descs:
        rc = lib.adi_wave_init(ctypes.byref(h), ctypes.byref(d), 1, one, one, None, None, None)
        assert rc == _lib.ADI_EINVAL
    d = _lib.Desc(10, 10, 1.0, 1.0, 0.01, 0, 0)
    assert lib.adi_wave_init(None, ctypes.byref(d), 1, one, one, None, None, None) == _lib.ADI_EINVAL
    assert lib.adi_wave_init(ctypes.byref(h), ctypes.byref(d), 0, one, one, None, None, None) == _lib.ADI_EINVAL
    nul = (ctypes.c_void_p * 1)(0)
    assert lib.adi_wave_init(ctypes.byref(h), ctypes.byref(d), 1, nul, one, None, None, None) == _lib.ADI_EINVAL
    src = (_lib.Source * 1)(_lib.Source(10, 0, 1, 5))  # ix outside the grid
    assert lib.adi_wave_init(ctypes.byref(h), ctypes.byref(d), 1, one, one, None, src, None) == _lib.ADI_EINVAL


def test_null_handle_calls_are_rejected(lib):
    assert lib.adi_wave_step(None, None, None) == _lib.ADI_EINVAL
    assert lib.adi_wave_run(None, 1, None, None, 0, None, None) == _lib.ADI_EINVAL
    assert lib.adi_wave_adjoint(None, None, None, None, 0, None) == _lib.ADI_EINVAL
    assert lib.adi_wave_sync_status(None, None) == _lib.ADI_EINVAL
    lib.adi_wave_destroy(None)


def test_step_noalloc_rejects_bad_arguments_without_gpu(lib):
    """adi_wave_step_noalloc checks every argument before its first CUDA call;
    the pointers here are never dereferenced (each call fails a check)."""
    f = lib.adi_wave_step_noalloc
    ok = _lib.Desc(100, 60, 1.0, 1.0, 0.001, 0, 0)
    m, uc, up = 0x10000, 0x20000, 0x30000  # 16-byte aligned, distinct
    EINVAL = _lib.ADI_EINVAL

    def call(desc=ok, ld=128, m_max=1.0, m_=m, uc_=uc, up_=up, src=None, k=1):
        return f(ctypes.byref(desc) if desc is not None else None, ld, m_max, m_, uc_, up_,
                 src, k, None)

    assert call(desc=None) == EINVAL
    assert call(m_=None) == EINVAL and call(uc_=None) == EINVAL and call(up_=None) == EINVAL
    assert call(desc=_lib.Desc(0, 60, 1.0, 1.0, 0.001, 0, 0)) == EINVAL       # nx < 1
    assert call(desc=_lib.Desc(100, 60, 1.0, 1.0, 0.0, 0, 0)) == EINVAL       # dt <= 0
    assert call(desc=_lib.Desc(100, 60, float("nan"), 1.0, 0.001, 0, 0)) == EINVAL
    assert call(desc=_lib.Desc(100, 60, 1.0, 1.0, 0.001, 0, 7)) == EINVAL     # fp64 mode
    assert call(ld=96) == EINVAL                                               # ld < nx
    assert call(ld=130) == EINVAL                                              # not a multiple of 32
    assert call(desc=_lib.Desc(4096, 2048, 1.0, 1.0, 0.001, 0, 0), ld=4096) == EINVAL  # > 2^22 floats
    assert call(m_max=0.0) == EINVAL and call(m_max=float("inf")) == EINVAL
    assert call(m_=m + 4) == EINVAL                                            # unaligned
    assert call(up_=uc) == EINVAL                                              # aliasing
    assert call(k=-1) == EINVAL
    src = _lib.Source(100, 10, 0x40000, 5)                                     # ix outside
    assert call(src=ctypes.byref(src)) == EINVAL
    assert b"source" in lib.adi_wave_last_error(None)
