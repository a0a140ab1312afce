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

    def set_model(self, scheme: str = "factored", g: Optional[torch.Tensor] = None,
                  f: Optional[torch.Tensor] = None):
        """adi_wave_set_model: scheme "factored" (Eq. CN1 in delta form; with g,
        the coefficient m^k = g[k] m, and with f [n_f, ny, nx], a source field
        f^k), "half_levels" (Eqs. fr1/fr2 as printed, over half time levels) or
        "listing1" (Listing 1's systems over half levels).  g and f are kept
        alive by the handle."""
        schemes = {"factored": 0, "half_levels": 1, "listing1": 2}
        if scheme not in schemes:
            raise ValueError("scheme must be one of %s" % sorted(schemes))
        if g is not None:
            g = _dev_f32(g, "g")
        if f is not None:
            f = _dev_f32(f, "f")
            if f.dim() != 3 or tuple(f.shape[1:]) != (self.ny, self.nx):
                raise ValueError("f must be [n_f, %d, %d]" % (self.ny, self.nx))
        mdl = _lib.Model(schemes[scheme], g.data_ptr() if g is not None else None,
                         int(g.numel()) if g is not None else 0,
                         f.data_ptr() if f is not None else None,
                         int(f.shape[0]) if f is not None else 0)
        _lib.check(self._lib.adi_wave_set_model(self._h, ctypes.byref(mdl)), self._h, "set_model")
        self._model_keep = [g, f]

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


class AdiWaveBatch:
    """Many independent grids ("shots") of uneven size advanced together.

    ``ms``, ``phis`` (and optional ``psis``): lists of float32 CUDA tensors
    [ny_b, nx_b]; ``dts``: tau per shot (a float applies to all).  Each step of
    all shots is one persistent kernel launch (``mode=0``) or the plain
    kernels launched per shot (``mode=1``).
    """

    def __init__(self, ms: Sequence[torch.Tensor], phis: Sequence[torch.Tensor], dts,
                 psis=None, start: str = "paper", fp64: str = "auto", stream=None):
        self._lib = _lib.load()
        n = len(ms)
        if n < 2 or len(phis) != n:
            raise ValueError("a batch needs >= 2 shots and one phi per m")
        if not isinstance(dts, (list, tuple)):
            dts = [dts] * n
        self.shapes = []
        keep = []
        descs = (Desc * n)()
        mp = (ctypes.c_void_p * n)()
        pp = (ctypes.c_void_p * n)()
        sp = (ctypes.c_void_p * n)()
        for b in range(n):
            ny, nx = phis[b].shape
            m = _dev_f32(ms[b], "m[%d]" % b, (ny, nx))
            phi = _dev_f32(phis[b], "phi[%d]" % b, (ny, nx))
            psi = _dev_f32(psis[b], "psi[%d]" % b, (ny, nx)) if psis and psis[b] is not None else None
            keep += [m, phi, psi]
            descs[b] = Desc(int(nx), int(ny), 1.0, 1.0, float(dts[b]), _START[start], _FP64[fp64])
            mp[b], pp[b] = m.data_ptr(), phi.data_ptr()
            sp[b] = psi.data_ptr() if psi is not None else 0
            self.shapes.append((int(ny), int(nx)))
        self.device = phis[0].device
        self._keep = keep
        h = ctypes.c_void_p()
        rc = self._lib.adi_wave_init(ctypes.byref(h), descs, n, mp, pp, sp, None, _stream_ptr(stream))
        _lib.check(rc, None, "adi_wave_init (batch)")
        self._h = h
        self.n = n

    def close(self):
        if getattr(self, "_h", None):
            self._lib.adi_wave_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_mode(self, mode: int):
        _lib.check(self._lib.adi_wave_set_batch_mode(self._h, int(mode)), self._h, "set_batch_mode")

    def set_wait_hook(self, spin_limit: int = 0, never_ready_shot: int = -1):
        _lib.check(self._lib.adi_wave_set_wait_hook(self._h, int(spin_limit), int(never_ready_shot)),
                   self._h, "set_wait_hook")

    def run(self, steps: int, srcs=None, wavelets=None, stream=None):
        """srcs: list of (ix, iy) or None per shot; wavelets: list of device tensors."""
        arr = None
        if srcs is not None:
            arr = (Source * self.n)()
            self._wav_keep = []
            for b in range(self.n):
                if srcs[b] is None:
                    arr[b] = Source(-1, -1, None, 0)
                else:
                    w = _dev_f32(wavelets[b].reshape(-1), "wavelet[%d]" % b)
                    self._wav_keep.append(w)
                    arr[b] = Source(int(srcs[b][0]), int(srcs[b][1]), w.data_ptr(), int(w.numel()))
        rc = self._lib.adi_wave_run(self._h, int(steps), arr, None, 0, ctypes.c_void_p(0),
                                    _stream_ptr(stream))
        _lib.check(rc, self._h, "run (batch)")

    def state(self, shot: int, stream=None):
        ny, nx = self.shapes[shot]
        up = torch.empty((ny, nx), dtype=torch.float32, device=self.device)
        uc = torch.empty_like(up)
        k = ctypes.c_int64()
        rc = self._lib.adi_wave_get_state(self._h, int(shot), _ptr(up), _ptr(uc), ctypes.byref(k),
                                          _stream_ptr(stream))
        _lib.check(rc, self._h, "get_state")
        return up, uc, int(k.value)

    def sync_status(self, stream=None):
        _lib.check(self._lib.adi_wave_sync_status(self._h, _stream_ptr(stream)), self._h,
                   "sync_status")

    def profile(self, enable: bool = True):
        _lib.check(self._lib.adi_wave_profile(self._h, int(bool(enable))), self._h)

    def profile_read(self):
        ms = (ctypes.c_double * _lib.ADI_KERNEL_KINDS)()
        cnt = (ctypes.c_int64 * _lib.ADI_KERNEL_KINDS)()
        _lib.check(self._lib.adi_wave_profile_read(self._h, ms, cnt, _lib.ADI_KERNEL_KINDS), self._h)
        return list(ms), list(cnt)

    def reset(self, phis: Sequence[torch.Tensor], ms=None, stream=None):
        """Re-run the start-up (Eq. CN2) of every shot in place."""
        n = self.n
        pp = (ctypes.c_void_p * n)()
        mp = (ctypes.c_void_p * n)() if ms is not None else None
        keep = []
        for b in range(n):
            phi = _dev_f32(phis[b], "phi[%d]" % b, self.shapes[b])
            keep.append(phi)
            pp[b] = phi.data_ptr()
            if ms is not None:
                m = _dev_f32(ms[b], "m[%d]" % b, self.shapes[b])
                keep.append(m)
                mp[b] = m.data_ptr()
        self._keep = keep
        rc = self._lib.adi_wave_reset(self._h, mp, pp, None, None, _stream_ptr(stream))
        _lib.check(rc, self._h, "reset (batch)")

    def launch_count(self) -> int:
        return int(self._lib.adi_wave_launch_count(self._h))


def step_noalloc(m: torch.Tensor, u_cur: torch.Tensor, u_prev: torch.Tensor, nx: int, dt: float,
                 m_max: float, k: int, lx: float = 1.0, ly: float = 1.0, fp64: str = "auto",
                 src: Optional[Tuple[int, int]] = None, wavelet: Optional[torch.Tensor] = None,
                 stream=None):
    """adi_wave_step_noalloc: one step on caller-owned PITCHED buffers.

    m, u_cur, u_prev are contiguous float32 CUDA tensors of shape [ny, ld]
    (ld a multiple of 32, >= nx, padding columns zero); u_prev is overwritten
    with u^{k+1}.  Neither this function nor the library call allocates
    device memory: the tensors are passed as they are (no copies), and the
    x sweep's intermediate lives in the library's fixed static array, which
    limits ld * ny to 4194304.  Calls on one device must not overlap.
    """
    lib = _lib.load()
    ny, ld = u_cur.shape
    for name, t in (("m", m), ("u_cur", u_cur), ("u_prev", u_prev)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32):
            raise TypeError("%s must be a float32 CUDA tensor" % name)
        if tuple(t.shape) != (ny, ld) or not t.is_contiguous():
            raise ValueError("%s must be a contiguous [%d, %d] tensor" % (name, ny, ld))
    srcs = None
    if src is not None:
        if wavelet is None or not wavelet.is_cuda or wavelet.dtype != torch.float32 \
                or not wavelet.is_contiguous():
            raise ValueError("a source needs contiguous float32 CUDA wavelet samples")
        srcs = Source(int(src[0]), int(src[1]), wavelet.data_ptr(), int(wavelet.numel()))
    desc = Desc(int(nx), int(ny), float(lx), float(ly), float(dt), 0, _FP64[fp64])
    with torch.cuda.device(u_cur.device):
        rc = lib.adi_wave_step_noalloc(ctypes.byref(desc), int(ld), float(m_max), _ptr(m),
                                       _ptr(u_cur), _ptr(u_prev),
                                       ctypes.byref(srcs) if srcs is not None else None, int(k),
                                       _stream_ptr(stream))
    _lib.check(rc, None, "adi_wave_step_noalloc")


def version() -> str:
    return _lib.load().adi_wave_version().decode()
