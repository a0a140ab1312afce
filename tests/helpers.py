"""Shared helpers for the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded FP32 inputs."""
import os

import numpy as np

import oracle

THREADS = os.cpu_count() or 1


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def smooth_state(nx, ny, seed, amp=1.0):
    """A smooth random field (sum of a few sine modes) for initial states."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 1.0) / (nx + 1)
    y = (np.arange(ny) + 1.0) / (ny + 1)
    u = np.zeros((ny, nx))
    for _ in range(4):
        p, q = rng.integers(1, 6, size=2)
        u += rng.standard_normal() * np.outer(np.sin(q * np.pi * y), np.sin(p * np.pi * x))
    return amp * u


def gpu_run(m, phi, tau, steps, psi=None, src=None, wavelet=None, rec=None, start="paper",
            fp64="auto", tuning=None, lx=1.0, ly=1.0, profile=False):
    """Returns dict(u_prev, u_cur, k, traces, handle_tuning) from the CUDA path."""
    import torch
    from paper_2006_10142_gb300 import api
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(f32(a)).to(dev)
    wav_t = t(wavelet) if wavelet is not None else None
    h = api.AdiWave(t(m), t(phi), tau, psi=t(psi) if psi is not None else None, lx=lx, ly=ly,
                    start=start, fp64=fp64, src=src, wavelet=wav_t)
    if tuning:
        h.set_tuning(**tuning)
    if profile:
        h.profile(True)
    traces = h.run(steps, src=src, wavelet=wav_t, rec=rec) if steps > 0 else None
    up, uc, k = h.state()
    h.sync_status()
    out = dict(u_prev=up.double().cpu().numpy(), u_cur=uc.double().cpu().numpy(), k=k,
               traces=None if traces is None else traces.double().cpu().numpy(),
               tuning=h.tuning(), handle=h)
    return out


def oracle_run(m, phi, tau, steps, psi=None, src=None, wavelet=None, rec=None, start="paper",
               lx=1.0, ly=1.0):
    """Same run in FP64 from the FP32-rounded inputs."""
    m64 = f32(m).astype(np.float64)
    phi64 = f32(phi).astype(np.float64)
    psi64 = f32(psi).astype(np.float64) if psi is not None else None
    wav64 = f32(wavelet).astype(np.float64) if wavelet is not None else None
    ny, nx = phi64.shape
    hx, hy = lx / (nx + 1), ly / (ny + 1)
    u0, u1 = oracle.adi_init(m64, phi64, hx, hy, tau, psi=psi64, taylor=(start == "taylor2"),
                             wv0=(wav64[0] if wav64 is not None else 0.0), src=src)
    up, uc, tr = oracle.adi_run(m64, u0, u1, hx, hy, tau, steps, k0=1, src=src, wavelet=wav64,
                                rec=rec, threads=THREADS)
    return dict(u_prev=up, u_cur=uc, traces=tr)
