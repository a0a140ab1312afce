"""Parity at the full workload sizes, over the whole run, in the launch
configuration the benchmark times (the planner's plan, autotuned as in
bench.py).

  - ricker_4096: 4096^2, 1000 time steps; ricker_16384: 16384^2, 200 time
    steps (Section 4's grid sizes, the factored scheme of Eq. CN1 split as
    Eqs. fr1/fr2).  The GPU run goes through the C ABI (adi_wave_run); the
    FP64 oracle runs the same number of steps from the same FP32-rounded
    inputs on all host threads.  Both final fields u^S and u^{S+1} must agree
    within relative L2 1e-4.
  - the step map itself: one step from the GPU's own final state
    (u^{k-1}, u^k), recomputed by the oracle in FP64, against the GPU's next
    step.
"""

import numpy as np
import pytest

from paper_2006_10142_gb300 import inputs
from helpers import THREADS, f32, rel_l2

import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _gpu_handle(prob, tune=True):
    import torch
    from paper_2006_10142_gb300 import api, autotune
    dev = torch.device("cuda:0")
    m = torch.from_numpy(f32(prob.m)).to(dev)
    phi = torch.zeros_like(m)
    wav = torch.from_numpy(f32(prob.wavelet)).to(dev)
    h = api.AdiWave(m, phi, prob.tau, src=prob.src, wavelet=wav)
    if tune:
        autotune.apply(h, steps=2, warmup=1)
        h.reset(phi)
    return h, wav


def _one_step_parity(h, prob, wav):
    up, uc, k = h.state()
    h.step(src=prob.src, wavelet=wav)
    _, un, k2 = h.state()
    assert k2 == k + 1
    n = prob.n
    hx = 1.0 / (n + 1)
    wv = float(f32(prob.wavelet)[k]) if k < len(prob.wavelet) else 0.0
    ref = oracle.adi_step(f32(prob.m).astype(np.float64), up.double().cpu().numpy(),
                          uc.double().cpu().numpy(), hx, hx, prob.tau, wv=wv, src=prob.src,
                          threads=THREADS)
    got = un.double().cpu().numpy()
    # the increment z = u^{k+1} - 2u^k + u^{k-1} is what the step computes; seen
    # through the FP32-stored u^{k+1} it carries that field's rounding, so its
    # error is measured against eps32 |u^{k+1}| as well as |z|
    z_ref = ref - 2 * uc.double().cpu().numpy() + up.double().cpu().numpy()
    z_got = got - 2 * uc.double().cpu().numpy() + up.double().cpu().numpy()
    scale = 1e-4 * np.linalg.norm(z_ref) + 8 * 2.0 ** -24 * np.linalg.norm(ref)
    return rel_l2(got, ref), float(np.linalg.norm(z_got - z_ref) / scale)


def _full_run_parity(n, steps):
    prob = inputs.ricker_problem(n, steps, seed=0, m_dtype=np.float32)
    h, wav = _gpu_handle(prob)
    h.run(steps, src=prob.src, wavelet=wav)
    h.sync_status()
    up, uc, k = h.state()
    assert k == steps + 1
    got_prev = up.double().cpu().numpy()
    got_cur = uc.double().cpu().numpy()
    # the oracle's run of the same length from the same start (u^0 = u^1 = 0)
    m64 = f32(prob.m).astype(np.float64)
    hx = 1.0 / (n + 1)
    z0, z1 = np.zeros((n, n)), np.zeros((n, n))
    ref_prev, ref_cur, _ = oracle.adi_run(m64, z0, z1, hx, hx, prob.tau, steps, k0=1,
                                          src=prob.src,
                                          wavelet=f32(prob.wavelet).astype(np.float64),
                                          threads=THREADS)
    del m64, z0, z1
    assert np.linalg.norm(ref_cur) > 0 and np.all(np.isfinite(got_cur))
    e_prev = rel_l2(got_prev, ref_prev)
    e_cur = rel_l2(got_cur, ref_cur)
    del ref_prev, ref_cur, got_prev, got_cur
    assert e_prev < 1e-4 and e_cur < 1e-4, (e_prev, e_cur)
    # the step map from the GPU's own final state
    e_u, e_z = _one_step_parity(h, prob, wav)
    assert e_u < 1e-6 and e_z < 1.0, (e_u, e_z)
    h.close()
    return e_prev, e_cur


def test_ricker_4096_full_run_matches_oracle():
    """ricker_4096: 4096^2, 1000 steps, both final fields against the oracle."""
    _full_run_parity(4096, 1000)


def test_ricker_16384_full_run_matches_oracle():
    """ricker_16384 (the bandwidth case): 16384^2, 200 steps, both final fields
    against the oracle (about 14 GiB of FP64 host memory, a few minutes on the
    host cores)."""
    _full_run_parity(16384, 200)
