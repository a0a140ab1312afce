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
- ``adi_step_gen`` / ``adi_run_gen``: Eq. (CN1) with a time-dependent
                   coefficient m^k = g_k m(x, y) (the c(t) of Eq. f1) and a
                   source field f^k(x, y), in the same delta form and split.
- ``adi_step_halves`` / ``adi_run_halves``: the sub-problems of Eqs. (fr1),
                   (fr2) taken literally over half time levels (variant 1), and
                   the fully implicit systems of Listing 1 (variant 2), with
                   Algorithm 1's buffer rotation.
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
            lib.oracle_adi_step_gen.argtypes = [ci, ci, cd, cd, cd, D, cd, cd, D, D, D, cd, ci, ci,
                                                D, ci]
            lib.oracle_adi_step_halves.argtypes = [ci, ci, ci, cd, cd, cd, D, D, D, cd, cd, ci, ci,
                                                   D, D, ci]
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


def _level(arr, k, hold_last):
    """Sample k of a per-level array: beyond its end the last sample
    (hold_last) or zero."""
    if arr is None:
        return None
    if 0 <= k < len(arr):
        return arr[k]
    if hold_last and len(arr) > 0:
        return arr[-1]
    return None


def adi_step_gen(m, u_prev, u_cur, hx, hy, tau, g_prev=1.0, g_next=1.0, fk=None, wv=0.0,
                 src=None, threads=1):
    """One step of Eq. (CN1) with m^k = g_k m and a source field f^k (CN1
    weighs Lap u^{k+1} by m^{k+1}/2 and Lap u^{k-1} by m^{k-1}/2)."""
    m, u_prev, u_cur, fk = _f64(m), _f64(u_prev), _f64(u_cur), _f64(fk)
    ny, nx = u_cur.shape
    out = np.empty_like(u_cur)
    sx, sy = (-1, -1) if src is None else (int(src[0]), int(src[1]))
    rc = _load().oracle_adi_step_gen(nx, ny, hx, hy, tau, _dp(m), float(g_prev), float(g_next),
                                     _dp(u_prev), _dp(u_cur), _dp(fk), float(wv), sx, sy, _dp(out),
                                     int(threads))
    if rc:
        raise RuntimeError("oracle_adi_step_gen failed (%d)" % rc)
    return out


def adi_run_gen(m, u_prev, u_cur, hx, hy, tau, steps, k0=1, g=None, f=None, src=None,
                wavelet=None, rec=None, threads=1):
    """`steps` steps of adi_step_gen from level k0.  g[k] scales m at level
    k (levels past the end of g keep its last value; g = None is 1); f[k] is
    the source field of level k (zero past its end); wavelet[k] the point
    source.  Returns (u^{k0+steps-1}, u^{k0+steps}, traces)."""
    up, uc = _f64(u_prev).copy(), _f64(u_cur).copy()
    rec = None if rec is None else np.asarray(rec, dtype=np.int64).reshape(-1, 2)
    tr = np.zeros((steps, 0 if rec is None else rec.shape[0]))
    for s in range(steps):
        k = k0 + s
        gp = _level(g, k - 1, True)
        gn = _level(g, k + 1, True)
        fk = _level(f, k, False)
        wv = _level(wavelet, k, False)
        un = adi_step_gen(m, up, uc, hx, hy, tau, 1.0 if gp is None else gp,
                          1.0 if gn is None else gn, fk, 0.0 if wv is None else wv, src, threads)
        if rec is not None:
            tr[s] = un[rec[:, 1], rec[:, 0]]
        up, uc = uc, un
    return up, uc, tr


def adi_step_halves(variant, m, u_half_prev, u_cur, hx, hy, tau, wv_k=0.0, wv_half=0.0, src=None,
                    threads=1):
    """One step of the literal sub-schemes: (u^{k-1/2}, u^k) -> (u^{k+1/2},
    u^{k+1}); variant 1 = Eqs. (fr1)/(fr2), variant 2 = Listing 1's systems."""
    m, a, b = _f64(m), _f64(u_half_prev), _f64(u_cur)
    ny, nx = b.shape
    uh = np.empty_like(b)
    un = np.empty_like(b)
    sx, sy = (-1, -1) if src is None else (int(src[0]), int(src[1]))
    rc = _load().oracle_adi_step_halves(int(variant), nx, ny, hx, hy, tau, _dp(m), _dp(a), _dp(b),
                                        float(wv_k), float(wv_half), sx, sy, _dp(uh), _dp(un),
                                        int(threads))
    if rc:
        raise RuntimeError("oracle_adi_step_halves failed (%d)" % rc)
    return uh, un


def adi_run_halves(variant, m, u_half_prev, u_cur, hx, hy, tau, steps, k0=1, src=None,
                   wavelet=None, rec=None, threads=1):
    """`steps` steps of adi_step_halves from level k0 (state (u^{k0-1/2},
    u^{k0})).  The source at level k is wavelet[k]; at the half level k + 1/2
    the mean of wavelet[k] and wavelet[k + 1] (zero past the end).  Returns
    (u^{k0+steps-1/2}, u^{k0+steps}, traces of u^{k0+s+1})."""
    a, b = _f64(u_half_prev).copy(), _f64(u_cur).copy()
    rec = None if rec is None else np.asarray(rec, dtype=np.int64).reshape(-1, 2)
    tr = np.zeros((steps, 0 if rec is None else rec.shape[0]))
    for s in range(steps):
        k = k0 + s
        w0 = _level(wavelet, k, False)
        w1 = _level(wavelet, k + 1, False)
        w0 = 0.0 if w0 is None else float(w0)
        w1 = 0.0 if w1 is None else float(w1)
        a, b = adi_step_halves(variant, m, a, b, hx, hy, tau, w0, 0.5 * (w0 + w1), src, threads)
        if rec is not None:
            tr[s] = b[rec[:, 1], rec[:, 0]]
    return a, b, tr
