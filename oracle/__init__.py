"""FP64 CPU oracle for the factored ADI scheme (test infrastructure only).

This package is the checker, not the product.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  It shares no code with the CUDA library
``paper_2006_10142_gb300``: both sides receive the same seeded inputs and
nothing else.

The arithmetic lives in ``adi_oracle.c`` (plain C, FP64, Thomas algorithm per
line); this module compiles it with gcc on first use and exposes numpy
wrappers.  Each wrapper names the passage of the paper it follows:

- ``adi_step``:    Eq. (CN1) in delta form, split into the x and y
                   sub-problems of Eqs. (fr1)/(fr2), Section 2 and Section 4.
- ``adi_init``:    Eq. (CN2) start-up (optionally the second-order Taylor start).
- ``adi_run``:     the time loop of Algorithm 1.
- ``adi_adjoint``: reverse-mode derivative of the receiver misfit through the
                   scheme above (not in the paper; derived from it).
- ``thomas``:      one tridiagonal solve (the serial method the paper's cyclic
                   reduction parallelises, Section 3.1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "adi_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``adi_oracle.c`` into ``oracle/_build/liboracle.so`` (gcc, -O2, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.POINTER(ctypes.c_int)
            ci, cd, cl = ctypes.c_int, ctypes.c_double, ctypes.c_long
            lib.oracle_thomas.argtypes = [ci, D, D, D, D, D]
            lib.oracle_laplacian.argtypes = [ci, ci, cd, cd, D, D]
            lib.oracle_laplacian.restype = None
            lib.oracle_adi_step.argtypes = [ci, ci, cd, cd, cd, D, D, D, cd, ci, ci, D, D, D, D, ci]
            lib.oracle_adi_init.argtypes = [ci, ci, cd, cd, cd, D, D, D, ci, cd, ci, ci, D, D]
            lib.oracle_adi_run.argtypes = [ci, ci, cd, cd, cd, D, D, D, cl, ci, ci, ci, D, ci,
                                           I, I, ci, D, ci]
            lib.oracle_adi_adjoint.argtypes = [ci, ci, cd, cd, cd, D, D, D, cl, ci, ci, ci, D, ci,
                                               I, I, ci, D, ci, D, D, D, D, ci]
            lib.oracle_line_sweep.argtypes = [ci, ci, ci, ci, cd, cd, D, D, D, ci]
            lib.oracle_num_threads_available.argtypes = []
            _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(_load().oracle_num_threads_available())


def grid_steps(nx: int, ny: int, lx: float = 1.0, ly: float = 1.0):
    """h1 = l/N1, h2 = l/N2 with N = n + 1 intervals (Eq. f6, n interior nodes)."""
    return lx / (nx + 1), ly / (ny + 1)


def thomas(a, b, c, d):
    """Solve a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i (a_0, c_{n-1} ignored)."""
    a, b, c, d = (_f64(v) for v in (a, b, c, d))
    n = d.shape[0]
    x = np.zeros(n)
    rc = _load().oracle_thomas(n, _dp(a), _dp(b), _dp(c), _dp(d), _dp(x))
    if rc:
        raise RuntimeError("oracle_thomas failed (%d)" % rc)
    return x


def line_sweep(m, rhs, h, tau, axis, transposed=False):
    """Op^{-1} rhs for Op = X = I - S Lap_x (axis 1, along rows, h = h1) or
    Y = I - S Lap_y (axis 0, along columns, h = h2), S = diag(tau^2 m / 2),
    or for their transposes."""
    m, rhs = _f64(m), _f64(rhs)
    ny, nx = rhs.shape
    out = np.empty_like(rhs)
    rc = _load().oracle_line_sweep(0 if axis == 1 else 1, int(bool(transposed)), nx, ny,
                                   float(h), float(tau), _dp(m), _dp(rhs), _dp(out), 1)
    if rc:
        raise RuntimeError("oracle_line_sweep failed (%d)" % rc)
    return out


def laplacian(u, hx, hy):
    """Five-point Laplacian with the zero Dirichlet ring (Eq. CN1's operator)."""
    u = _f64(u)
    ny, nx = u.shape
    out = np.empty_like(u)
    _load().oracle_laplacian(nx, ny, hx, hy, _dp(u), _dp(out))
    return out


def adi_step(m, u_prev, u_cur, hx, hy, tau, wv=0.0, src=None, threads=1, return_parts=False):
    """One factored-ADI step u^{k-1}, u^k -> u^{k+1} (Eqs. CN1, fr1, fr2)."""
    m, u_prev, u_cur = _f64(m), _f64(u_prev), _f64(u_cur)
    ny, nx = u_cur.shape
    sx, sy = (-1, -1) if src is None else (int(src[0]), int(src[1]))
    out = np.empty_like(u_cur)
    r = np.empty_like(u_cur)
    w = np.empty_like(u_cur)
    z = np.empty_like(u_cur)
    rc = _load().oracle_adi_step(nx, ny, hx, hy, tau, _dp(m), _dp(u_prev), _dp(u_cur), float(wv),
                                 sx, sy, _dp(out), _dp(r), _dp(w), _dp(z), int(threads))
    if rc:
        raise RuntimeError("oracle_adi_step failed (%d)" % rc)
    if return_parts:
        return out, r, w, z
    return out


def adi_init(m, phi, hx, hy, tau, psi=None, taylor=False, wv0=0.0, src=None):
    """Start-up of Eq. (CN2): returns (u^0, u^1)."""
    m, phi, psi = _f64(m), _f64(phi), _f64(psi)
    ny, nx = phi.shape
    sx, sy = (-1, -1) if src is None else (int(src[0]), int(src[1]))
    u0 = np.empty_like(phi)
    u1 = np.empty_like(phi)
    _load().oracle_adi_init(nx, ny, hx, hy, tau, _dp(m), _dp(phi), _dp(psi), int(bool(taylor)),
                            float(wv0), sx, sy, _dp(u0), _dp(u1))
    return u0, u1


def adi_run(m, u_prev, u_cur, hx, hy, tau, steps, k0=1, src=None, wavelet=None, rec=None,
            threads=1):
    """Algorithm 1's time loop.  Returns (u_prev, u_cur, traces) after `steps` steps.

    ``src`` = (ix, iy) node of the point source, ``wavelet[k]`` = w(t_k) used
    by the step leaving level k; ``rec`` = int array [n_rec, 2] of (ix, iy);
    ``traces[s, r]`` = u^{k0+s+1} at receiver r.
    """
    m = _f64(m)
    up = _f64(u_prev).copy()
    uc = _f64(u_cur).copy()
    ny, nx = uc.shape
    sx, sy = (-1, -1) if src is None else (int(src[0]), int(src[1]))
    wav = _f64(wavelet) if wavelet is not None else None
    nw = 0 if wav is None else wav.shape[0]
    if rec is None:
        rec = np.zeros((0, 2), dtype=np.int32)
    rec = np.ascontiguousarray(rec, dtype=np.int32).reshape(-1, 2)
    rx = np.ascontiguousarray(rec[:, 0])
    ry = np.ascontiguousarray(rec[:, 1])
    nrec = rec.shape[0]
    traces = np.zeros((max(steps, 0), nrec))
    rc = _load().oracle_adi_run(nx, ny, hx, hy, tau, _dp(m), _dp(up), _dp(uc), int(k0), int(steps),
                                sx, sy, _dp(wav), nw, _ip(rx), _ip(ry), nrec, _dp(traces),
                                int(threads))
    if rc:
        raise RuntimeError("oracle_adi_run failed (%d)" % rc)
    return up, uc, traces


def adi_adjoint(m, u_prev0, u_cur0, hx, hy, tau, steps, resid, rec, k0=1, src=None,
                wavelet=None, taylor_k0=False, threads=1):
    """Reverse-mode gradient of J = 1/2 sum (traces - d)^2 with resid = traces - d.

    Returns dict(grad_m, grad_wavelet, lam_cur, lam_prev).
    """
    m, u_prev0, u_cur0 = _f64(m), _f64(u_prev0), _f64(u_cur0)
    ny, nx = u_cur0.shape
    sx, sy = (-1, -1) if src is None else (int(src[0]), int(src[1]))
    wav = _f64(wavelet) if wavelet is not None else None
    nw = 0 if wav is None else wav.shape[0]
    rec = np.ascontiguousarray(rec, dtype=np.int32).reshape(-1, 2)
    rx = np.ascontiguousarray(rec[:, 0])
    ry = np.ascontiguousarray(rec[:, 1])
    nrec = rec.shape[0]
    resid = _f64(resid).reshape(steps, nrec)
    gm = np.zeros_like(u_cur0)
    gw = np.zeros(nw) if nw else None
    lc = np.zeros_like(u_cur0)
    lp = np.zeros_like(u_cur0)
    rc = _load().oracle_adi_adjoint(nx, ny, hx, hy, tau, _dp(m), _dp(u_prev0), _dp(u_cur0),
                                    int(k0), int(steps), sx, sy, _dp(wav), nw, _ip(rx), _ip(ry),
                                    nrec, _dp(resid), int(bool(taylor_k0)), _dp(gm), _dp(gw),
                                    _dp(lc), _dp(lp), int(threads))
    if rc:
        raise RuntimeError("oracle_adi_adjoint failed (%d)" % rc)
    return {"grad_m": gm, "grad_wavelet": gw, "lam_cur": lc, "lam_prev": lp}
