"""torch.autograd integration (forward = run, backward = adjoint) and the
autotuner (every tuning it picks is timed and stays at oracle parity)."""
import math

import numpy as np
import pytest

import oracle
from paper_2006_10142_gb300 import inputs
from helpers import THREADS, f32, oracle_run, rel_l2, smooth_state

pytestmark = pytest.mark.gpu


def test_autograd_gradient_matches_oracle_adjoint():
    import torch
    from paper_2006_10142_gb300.autograd import simulate
    dev = torch.device("cuda:0")
    n, steps = 48, 90
    prob, m_true = inputs.adjoint_problem(n, steps, seed=3, n_rec=12)
    hx = 1.0 / (n + 1)
    z = np.zeros((n, n))
    _, _, d = oracle.adi_run(f32(m_true).astype(np.float64), z, z, hx, hx, prob.tau, steps,
                             src=prob.src, wavelet=f32(prob.wavelet).astype(np.float64),
                             rec=prob.rec, threads=THREADS)
    m = torch.tensor(f32(prob.m), device=dev, requires_grad=True)
    wav = torch.tensor(f32(prob.wavelet), device=dev, requires_grad=True)
    traces = simulate(m, wav, prob.src, prob.rec, steps, prob.tau, ckpt_every=10)
    loss = 0.5 * ((traces.double() - torch.from_numpy(d).to(dev)) ** 2).sum()
    loss.backward()
    resid = (traces.detach().double().cpu().numpy() - d)
    ref = oracle.adi_adjoint(f32(prob.m).astype(np.float64), z, z, hx, hx, prob.tau, steps,
                             resid, prob.rec, src=prob.src,
                             wavelet=f32(prob.wavelet).astype(np.float64), threads=THREADS)
    assert rel_l2(m.grad.double().cpu().numpy(), ref["grad_m"]) < 1e-4
    assert rel_l2(wav.grad.double().cpu().numpy(), ref["grad_wavelet"]) < 1e-4


def test_autograd_through_speed():
    """m = c^2 built in torch: autograd applies dJ/dc = 2c dJ/dm."""
    import torch
    from paper_2006_10142_gb300.autograd import simulate
    dev = torch.device("cuda:0")
    n, steps = 32, 40
    prob, _ = inputs.adjoint_problem(n, steps, seed=1, n_rec=8)
    c = torch.tensor(np.sqrt(f32(prob.m)), device=dev, requires_grad=True)
    wav = torch.tensor(f32(prob.wavelet), device=dev)
    traces = simulate(c * c, wav, prob.src, prob.rec, steps, prob.tau, ckpt_every=8)
    traces.pow(2).sum().mul(0.5).backward()
    gc = c.grad.clone()
    m = (c.detach() ** 2).requires_grad_(True)
    traces = simulate(m, wav, prob.src, prob.rec, steps, prob.tau, ckpt_every=8)
    traces.pow(2).sum().mul(0.5).backward()
    torch.testing.assert_close(gc, 2 * c.detach() * m.grad, rtol=1e-5, atol=1e-12)


def test_autotune_picks_valid_fast_tuning(tmp_path, monkeypatch):
    monkeypatch.setenv("ADIWAVE_TUNE_CACHE", str(tmp_path / "tune.json"))
    from paper_2006_10142_gb300 import autotune
    nx, ny = 700, 520
    res = autotune.tune(nx, ny, steps=2, warmup=1)
    assert res["x_ms"] > 0 and res["y_ms"] > 0
    again = autotune.tune(nx, ny)  # from the cache
    assert again == res
    # the chosen tuning is exact
    m = inputs.m_field(nx, ny, 0)
    tau = 0.5 / (max(nx, ny) + 1) / math.sqrt(m.max())
    phi = smooth_state(nx, ny, 2, 1e-2)
    from helpers import gpu_run
    g = gpu_run(m, phi, tau, 6, tuning=res["tuning"])
    o = oracle_run(m, phi, tau, 6)
    assert rel_l2(g["u_cur"], o["u_cur"]) < 1e-4
