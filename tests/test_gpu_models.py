"""GPU parity of the problem class beyond the workloads and of the paper's
literal sub-schemes (adi_wave_set_model) against the FP64 oracle.

- "factored" with g and f: Eq. (CN1) with the coefficient m^k = g_k m (the
  c(t) of Eq. f1) and a source field f^k, against oracle.adi_run_gen;
- "half_levels": Eqs. (fr1)/(fr2) as printed over half time levels, against
  oracle.adi_run_halves(1, ...) and the closed form of the standing mode
  (which turns about sqrt 2 too fast);
- "listing1": Listing 1's systems, against oracle.adi_run_halves(2, ...)
  (every mode decays).
Bar: relative L2 <= 1e-4 per field after the run, as for the default path.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2006_10142_gb300 import inputs
from helpers import THREADS, f32, rel_l2, smooth_state

pytestmark = pytest.mark.gpu
TOL = 1e-4


def _dev():
    import torch
    return torch.device("cuda:0")


def _problem(nx, ny, steps, seed, cfl=0.5):
    m = inputs.m_field(nx, ny, seed)
    h = min(1.0 / (nx + 1), 1.0 / (ny + 1))
    tau = cfl * h / math.sqrt(m.max())
    phi = smooth_state(nx, ny, seed, 1e-2)
    src = (nx // 3, (2 * ny) // 3)
    wav = inputs.wavelet_samples(steps + 2, tau, fp=3.0)
    rec = np.array([[i % nx, (5 * i + 1) % ny] for i in range(6)], dtype=np.int32)
    return m, phi, tau, src, wav, rec


def _gpu(m, phi, tau, steps, src, wav, rec, scheme, g=None, f=None):
    import torch
    from paper_2006_10142_gb300 import api
    dev = _dev()
    t = lambda a: torch.from_numpy(f32(a)).to(dev)
    wav_t = t(wav)
    h = api.AdiWave(t(m), t(phi), tau, src=src, wavelet=wav_t)
    h.set_model(scheme, g=t(g) if g is not None else None, f=t(f) if f is not None else None)
    tr = h.run(steps, src=src, wavelet=wav_t, rec=rec)
    up, uc, k = h.state()
    h.sync_status()
    out = (up.double().cpu().numpy(), uc.double().cpu().numpy(), k,
           None if tr is None else tr.double().cpu().numpy())
    h.close()
    return out


@pytest.mark.parametrize("nx,ny", [(37, 53), (300, 40), (129, 257), (40, 3000), (1000, 300)])
@pytest.mark.parametrize("variant,scheme", [(1, "half_levels"), (2, "listing1")])
def test_half_level_schemes_match_oracle(nx, ny, variant, scheme):
    steps = 10
    m, phi, tau, src, wav, rec = _problem(nx, ny, steps, seed=nx + ny + variant)
    up, uc, k, tr = _gpu(m, phi, tau, steps, src, wav, rec, scheme)
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    p64 = f32(phi).astype(np.float64)
    ra, rb, rtr = oracle.adi_run_halves(variant, f32(m).astype(np.float64), p64, p64, hx, hy, tau,
                                        steps, k0=1, src=src,
                                        wavelet=f32(wav).astype(np.float64), rec=rec,
                                        threads=THREADS)
    assert k == steps + 1
    assert rel_l2(up, ra) < TOL and rel_l2(uc, rb) < TOL, (rel_l2(up, ra), rel_l2(uc, rb))
    assert rel_l2(tr, rtr) < TOL


def test_half_levels_standing_mode_turns_sqrt2_too_fast():
    """c = 1, f = 0, u(0) = sin(pi x) sin(pi y): the GPU run of Eqs. fr1/fr2
    follows the mode's closed form a_q = cos((q - 1/2) theta) / cos(theta / 2)
    with cos theta = 1 / (1 + tau^2 P / 2) per half level, whose phase per
    step is about sqrt 2 times the wave's."""
    n, steps = 128, 200
    h = 1.0 / (n + 1)
    tau = h
    x = (np.arange(n) + 1.0) * h
    phi = np.outer(np.sin(np.pi * x), np.sin(np.pi * x))
    up, uc, _, _ = _gpu(np.ones((n, n)), phi, tau, steps, None, np.zeros(steps + 2), None,
                        "half_levels")
    P = 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    th = math.acos(1.0 / (1.0 + tau * tau * P / 2.0))
    amp = math.cos((2 * steps + 0.5) * th) / math.cos(th / 2)
    assert rel_l2(uc, amp * phi) < TOL
    assert 2 * th / (tau * math.sqrt(2 * P)) == pytest.approx(math.sqrt(2.0), rel=2e-3)


@pytest.mark.parametrize("nx,ny", [(37, 53), (300, 40), (129, 257), (40, 3000), (1000, 300)])
def test_time_dependent_coefficient_and_source_field_match_oracle(nx, ny):
    steps = 10
    m, phi, tau, src, wav, rec = _problem(nx, ny, steps, seed=3 * nx + ny)
    g = 1.0 + 0.3 * np.sin(0.37 * np.arange(steps + 4))
    rng = np.random.default_rng(nx)
    f = np.array([smooth_state(nx, ny, int(rng.integers(1 << 30)), 50.0) for _ in range(steps - 3)])
    up, uc, k, tr = _gpu(m, phi, tau, steps, src, wav, rec, "factored", g=g, f=f)
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    p64 = f32(phi).astype(np.float64)
    ra, rb, rtr = oracle.adi_run_gen(f32(m).astype(np.float64), p64, p64, hx, hy, tau, steps, k0=1,
                                     g=f32(g).astype(np.float64), f=f32(f).astype(np.float64),
                                     src=src, wavelet=f32(wav).astype(np.float64), rec=rec,
                                     threads=THREADS)
    assert k == steps + 1
    assert rel_l2(up, ra) < TOL and rel_l2(uc, rb) < TOL, (rel_l2(up, ra), rel_l2(uc, rb))
    assert rel_l2(tr, rtr) < TOL


def test_model_restrictions():
    import torch
    from paper_2006_10142_gb300 import _lib, api
    dev = _dev()
    m = torch.ones((20, 24), device=dev)
    h = api.AdiWave(m, torch.zeros_like(m), 0.01)
    with pytest.raises(_lib.AdiError) as ei:
        h.set_model("half_levels", g=torch.ones(4, device=dev))
    assert ei.value.code == _lib.ADI_EINVAL
    h.set_model("factored", g=torch.ones(4, device=dev))
    h.set_checkpointing(2)
    tr = h.run(4, rec=np.array([[3, 3]], dtype=np.int32))
    with pytest.raises(_lib.AdiError) as ei:
        h.adjoint(torch.zeros_like(tr))
    assert ei.value.code == _lib.ADI_EUNSUPPORTED
    # the default model restores the default path (graph replay, adjoint)
    h.set_model("factored")
    tr = h.run(4, rec=np.array([[3, 3]], dtype=np.int32))
    h.adjoint(torch.zeros_like(tr))
    h.sync_status()
    h.close()
    B = api.AdiWaveBatch([m, m], [torch.zeros_like(m)] * 2, [0.01, 0.01])
    with pytest.raises(_lib.AdiError) as ei:
        _lib.check(B._lib.adi_wave_set_model(B._h, __import__("ctypes").byref(_lib.Model(1, None, 0, None, 0))),
                   B._h, "set_model")
    assert ei.value.code == _lib.ADI_EUNSUPPORTED
    B.close()
