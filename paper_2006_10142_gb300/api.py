"""Python binding of the C ABI (include/adiwave.h), on top of PyTorch tensors.

PyTorch supplies device memory and the CUDA stream; every step of the
computation runs in libadiwave.so.  Tensors are FP32, contiguous, shape
[ny, nx] (x fastest), on a CUDA device; grid conventions follow Section 2,
Eq. (f6): nx x ny interior nodes of the domain [0, lx] x [0, ly].
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence, Tuple

import torch

from . import _lib
from ._lib import AdiError, Desc, Source, Tuning  # noqa: F401

_START = {"paper": _lib.ADI_START_PAPER, "taylor2": _lib.ADI_START_TAYLOR2}
_FP64 = {"auto": _lib.ADI_FP64_AUTO, "never": _lib.ADI_FP64_NEVER, "always": _lib.ADI_FP64_ALWAYS}


def _stream_ptr(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev_f32(t: torch.Tensor, name: str, shape=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch.Tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float32:
        raise TypeError("%s must be float32" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    return t.contiguous()


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


class AdiWave:
    """One grid advanced by the factored ADI scheme (Eqs. CN1, CN2, fr1, fr2).

    m    = c^2 coefficient [ny, nx] (> 0), phi = u(0), psi = u_t(0) (optional);
    dt   = tau; src = (ix, iy) point-source node with wavelet samples
    ``wavelet[k] = w(t_k)`` (device float32) -- used by the Taylor start only
    at init and by every step when passed to run()/step().
    """

    def __init__(self, m: torch.Tensor, phi: torch.Tensor, dt: float,
                 psi: Optional[torch.Tensor] = None, lx: float = 1.0, ly: float = 1.0,
                 start: str = "paper", fp64: str = "auto",
                 src: Optional[Tuple[int, int]] = None, wavelet: Optional[torch.Tensor] = None,
                 stream=None):
        self._lib = _lib.load()
        ny, nx = phi.shape
        m = _dev_f32(m, "m", (ny, nx))
        phi = _dev_f32(phi, "phi", (ny, nx))
        psi = _dev_f32(psi, "psi", (ny, nx)) if psi is not None else None
        self.nx, self.ny, self.dt, self.lx, self.ly = int(nx), int(ny), float(dt), lx, ly
        self.device = phi.device
        desc = Desc(self.nx, self.ny, float(lx), float(ly), float(dt), _START[start], _FP64[fp64])
        self._keep = [m, phi, psi]
        srcs = self._sources(src, wavelet)
        h = ctypes.c_void_p()
        mp = (ctypes.c_void_p * 1)(m.data_ptr())
        pp = (ctypes.c_void_p * 1)(phi.data_ptr())
        sp = (ctypes.c_void_p * 1)(psi.data_ptr() if psi is not None else 0)
        with torch.cuda.device(self.device):
            rc = self._lib.adi_wave_init(ctypes.byref(h), ctypes.byref(desc), 1, mp, pp, sp,
                                         srcs, _stream_ptr(stream))
        _lib.check(rc, None, "adi_wave_init")
        self._h = h
        self._run_keep = []

    # -- helpers ---------------------------------------------------------------
    def _sources(self, src, wavelet):
        if src is None:
            return None
        if wavelet is None:
            raise ValueError("a source needs wavelet samples")
        wavelet = _dev_f32(wavelet.reshape(-1), "wavelet")
        self._wav_keep = wavelet
        arr = (Source * 1)()
        arr[0] = Source(int(src[0]), int(src[1]), wavelet.data_ptr(), int(wavelet.numel()))
        return arr

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.adi_wave_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, phi: torch.Tensor, m: Optional[torch.Tensor] = None,
              psi: Optional[torch.Tensor] = None, src=None, wavelet=None, stream=None):
        """Re-run the start-up (Eq. CN2) in place, optionally with a new m."""
        shape = (self.ny, self.nx)
        phi = _dev_f32(phi, "phi", shape)
        m = _dev_f32(m, "m", shape) if m is not None else None
        psi = _dev_f32(psi, "psi", shape) if psi is not None else None
        srcs = self._sources(src, wavelet)
        mp = (ctypes.c_void_p * 1)(m.data_ptr()) if m is not None else None
        pp = (ctypes.c_void_p * 1)(phi.data_ptr())
        sp = (ctypes.c_void_p * 1)(psi.data_ptr()) if psi is not None else None
        self._keep = [m, phi, psi]
        rc = self._lib.adi_wave_reset(self._h, mp, pp, sp, srcs, _stream_ptr(stream))
        _lib.check(rc, self._h, "reset")

    # -- time stepping -----------------------------------------------------------
    def step(self, src=None, wavelet=None, stream=None):
        srcs = self._sources(src, wavelet)
        _lib.check(self._lib.adi_wave_step(self._h, srcs, _stream_ptr(stream)), self._h, "step")

    def run(self, steps: int, src=None, wavelet=None, rec=None, stream=None):
        """Advance `steps` steps; returns traces [steps, n_rec] (or None)."""
        srcs = self._sources(src, wavelet)
        traces = None
        rec_arr = None
        n_rec = 0
        if rec is not None:
            import numpy as np
            r = np.ascontiguousarray(np.asarray(rec, dtype=np.int32).reshape(-1, 2))
            n_rec = r.shape[0]
            rec_arr = (ctypes.c_int32 * (2 * n_rec))(*r.ravel().tolist())
            traces = torch.zeros((steps, n_rec), dtype=torch.float32, device=self.device)
        self._run_keep = [srcs, getattr(self, "_wav_keep", None), traces]
        rc = self._lib.adi_wave_run(self._h, int(steps), srcs, rec_arr, n_rec, _ptr(traces),
                                    _stream_ptr(stream))
        _lib.check(rc, self._h, "run")
        return traces

    def set_checkpointing(self, every: int):
        _lib.check(self._lib.adi_wave_set_checkpointing(self._h, int(every)), self._h)

    def adjoint(self, resid: torch.Tensor, ckpt_every: int = 0, want_wavelet: bool = True,
                stream=None):
        """dJ/dm (float64 [ny, nx]) and dJ/dwavelet for the last run, resid = traces - data."""
        resid = _dev_f32(resid, "resid")
        gm = torch.zeros((self.ny, self.nx), dtype=torch.float64, device=self.device)
        wav = getattr(self, "_wav_keep", None)
        gw = torch.zeros_like(wav) if (want_wavelet and wav is not None) else None
        rc = self._lib.adi_wave_adjoint(self._h, _ptr(resid), _ptr(gm), _ptr(gw), int(ckpt_every),
                                        _stream_ptr(stream))
        _lib.check(rc, self._h, "adjoint")
        return gm, gw

    # -- state -------------------------------------------------------------------
    def state(self, stream=None):
        up = torch.empty((self.ny, self.nx), dtype=torch.float32, device=self.device)
        uc = torch.empty_like(up)
        k = ctypes.c_int64()
        rc = self._lib.adi_wave_get_state(self._h, 0, _ptr(up), _ptr(uc), ctypes.byref(k),
                                          _stream_ptr(stream))
        _lib.check(rc, self._h, "get_state")
        return up, uc, int(k.value)

    def set_state(self, u_prev: torch.Tensor, u_cur: torch.Tensor, k: int, stream=None):
        u_prev = _dev_f32(u_prev, "u_prev", (self.ny, self.nx))
        u_cur = _dev_f32(u_cur, "u_cur", (self.ny, self.nx))
        rc = self._lib.adi_wave_set_state(self._h, 0, _ptr(u_prev), _ptr(u_cur), int(k),
                                          _stream_ptr(stream))
        _lib.check(rc, self._h, "set_state")

    def sync_status(self, stream=None):
        rc = self._lib.adi_wave_sync_status(self._h, _stream_ptr(stream))
        _lib.check(rc, self._h, "sync_status")

    # -- tuning / measurement -------------------------------------------------------
    def tuning(self) -> dict:
        t = Tuning()
        _lib.check(self._lib.adi_wave_get_tuning(self._h, ctypes.byref(t)), self._h)
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def set_tuning(self, **kw):
        t = Tuning(**{f: int(kw.get(f, 0)) for f, _ in Tuning._fields_})
        _lib.check(self._lib.adi_wave_set_tuning(self._h, ctypes.byref(t)), self._h, "set_tuning")

    def profile(self, enable: bool = True):
        _lib.check(self._lib.adi_wave_profile(self._h, int(bool(enable))), self._h)

    def profile_read(self):
        ms = (ctypes.c_double * _lib.ADI_KERNEL_KINDS)()
        cnt = (ctypes.c_int64 * _lib.ADI_KERNEL_KINDS)()
        _lib.check(self._lib.adi_wave_profile_read(self._h, ms, cnt, _lib.ADI_KERNEL_KINDS), self._h)
        return list(ms), list(cnt)

    def launch_count(self) -> int:
        return int(self._lib.adi_wave_launch_count(self._h))


def version() -> str:
    return _lib.load().adi_wave_version().decode()
