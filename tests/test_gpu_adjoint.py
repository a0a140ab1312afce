"""GPU adjoint (C ABI adi_wave_adjoint) against the FP64 oracle adjoint and
against finite differences of the GPU forward run.

Every case uses the adjoint workload's recipe (seeded c-field,
tau = 0.5 h / max c, Ricker source at (0.5, 0.9), 64 receivers along
y = 0.1).  Residuals handed to both sides come from the oracle's traces or
from a seeded generator, never from the GPU's.  Bars: dJ/dm and dJ/dwavelet
within relative L2 1e-4 of the FP64 oracle adjoint; at 1024^2 x 2000 steps
(checkpoint every 50) also the directional derivative against central
differences of the GPU misfit within 1e-2 in 16 seeded directions.
"""

import numpy as np
import pytest

import oracle
from paper_2006_10142_gb300 import inputs
from helpers import THREADS, f32, rel_l2

pytestmark = pytest.mark.gpu


def _dev():
    import torch
    return torch.device("cuda:0")


def _oracle_traces(prob, m, u0=None, u1=None, k0=1):
    n = prob.n
    hx = 1.0 / (n + 1)
    z = np.zeros((n, n))
    u0 = z if u0 is None else u0
    u1 = z if u1 is None else u1
    _, _, tr = oracle.adi_run(f32(m).astype(np.float64), u0, u1, hx, hx, prob.tau, prob.steps,
                              k0=k0, src=prob.src, wavelet=f32(prob.wavelet).astype(np.float64),
                              rec=prob.rec, threads=THREADS)
    return tr


def _oracle_grad(prob, m, resid, u0, u1, k0=1, start="paper"):
    n = prob.n
    hx = 1.0 / (n + 1)
    return oracle.adi_adjoint(f32(m).astype(np.float64), u0, u1, hx, hx, prob.tau, prob.steps,
                              np.asarray(resid, dtype=np.float64), prob.rec, k0=k0, src=prob.src,
                              wavelet=f32(prob.wavelet).astype(np.float64),
                              taylor_k0=(start == "taylor2"), threads=THREADS)


def _gpu_grad(prob, every, resid, u_prev=None, u_cur=None, k0=1, tuning=None, phi=None,
              start="paper"):
    """GPU forward run (checkpoints every `every`) and gradient; returns
    (traces, grad_m, grad_wavelet), or None when `tuning` does not fit."""
    import torch
    from paper_2006_10142_gb300 import _lib, api
    dev = _dev()
    n = prob.n
    wav = torch.from_numpy(f32(prob.wavelet)).to(dev)
    phi_t = torch.from_numpy(f32(phi if phi is not None else np.zeros((n, n)))).to(dev)
    h = api.AdiWave(torch.from_numpy(f32(prob.m)).to(dev), phi_t, prob.tau, start=start,
                    src=prob.src, wavelet=wav)
    try:
        if tuning:
            try:
                h.set_tuning(**tuning)
            except _lib.AdiError as e:
                assert e.code == _lib.ADI_EUNSUPPORTED, str(e)
                return None
            got = h.tuning()
            assert all(got[k] == v for k, v in tuning.items()), (got, tuning)
        if u_prev is not None:
            h.set_state(torch.from_numpy(f32(u_prev)).to(dev), torch.from_numpy(f32(u_cur)).to(dev),
                        k0)
        h.set_checkpointing(every)
        tr = h.run(prob.steps, src=prob.src, wavelet=wav, rec=prob.rec)
        gm, gw = h.adjoint(torch.from_numpy(f32(resid)).to(dev))
        h.sync_status()
        return tr.double().cpu().numpy(), gm.cpu().numpy(), gw.double().cpu().numpy()
    finally:
        h.close()


@pytest.mark.parametrize("every", [1, 7, 50, 150])
def test_adjoint_matches_fp64_oracle(every):
    """64^2, 150 steps of the adjoint recipe; residual = oracle traces of m
    minus oracle data of the perturbed medium."""
    prob, m_true = inputs.adjoint_problem(64, 150, seed=2, n_rec=16)
    d = _oracle_traces(prob, m_true)
    tr_ref = _oracle_traces(prob, prob.m)
    resid = f32(tr_ref - d)
    z = np.zeros((64, 64))
    ref = _oracle_grad(prob, prob.m, resid, z, z)
    tr, gm, gw = _gpu_grad(prob, every, resid)
    assert rel_l2(tr, tr_ref) < 1e-4
    e_m = rel_l2(gm, ref["grad_m"])
    e_w = rel_l2(gw, ref["grad_wavelet"])
    assert e_m < 1e-4 and e_w < 1e-4, (e_m, e_w)


# ---------------------------------------------------------------------------
# windows of the adjoint recipe on ragged grids
# ---------------------------------------------------------------------------
WINDOW_STEPS = 40
_WINDOW_CACHE = {}


def _recipe_window(n):
    """A 40-step window of the adjoint recipe on an n x n grid, starting when
    the source's wave has reached the receivers (t = 0.45): the start state
    (u^{k0-1}, u^{k0}) is the oracle's run of the recipe from rest, rounded to
    FP32 (an input of both sides); residuals are seeded, standard deviation
    1e-2.  Within 40 steps the receivers' adjoint field reaches the source
    only through the implicit solves' exponential tails, so dJ/dwavelet is
    near underflow here: the windows compare dJ/dm, the runs from rest
    (64^2, 1024^2) both gradients."""
    if n in _WINDOW_CACHE:
        return _WINDOW_CACHE[n]
    base, _ = inputs.adjoint_problem(n, WINDOW_STEPS, seed=0, n_rec=64)
    s0 = int(round(0.45 / base.tau))
    prob = inputs.ricker_problem(n, s0 + WINDOW_STEPS, seed=0, src=base.src)
    prob.rec = base.rec
    hx = 1.0 / (n + 1)
    z = np.zeros((n, n))
    up, uc, _ = oracle.adi_run(f32(prob.m).astype(np.float64), z, z, hx, hx, prob.tau, s0, k0=1,
                               src=prob.src, wavelet=f32(prob.wavelet).astype(np.float64),
                               threads=THREADS)
    prob.steps = WINDOW_STEPS
    rng = np.random.default_rng(n)
    resid = f32(1e-2 * rng.standard_normal((WINDOW_STEPS, prob.rec.shape[0])))
    out = (prob, f32(up), f32(uc), 1 + s0, resid)
    _WINDOW_CACHE[n] = out
    return out


def _window_parity(n, **tuning):
    prob, up, uc, k0, resid = _recipe_window(n)
    r = _gpu_grad(prob, 10, resid, u_prev=up, u_cur=uc, k0=k0, tuning=tuning)
    if r is None:
        return None
    _, gm, _ = r
    ref = _oracle_grad(prob, prob.m, resid, up.astype(np.float64), uc.astype(np.float64), k0=k0)
    assert np.linalg.norm(ref["grad_m"]) > 0
    return rel_l2(gm, ref["grad_m"])


@pytest.mark.parametrize("n,ky,ty", [(300, 16, 256), (300, 32, 512), (700, 32, 256),
                                     (1000, 32, 256)])
@pytest.mark.parametrize("ys", [2, 3, 4])
def test_adjoint_column_solve_forms_match_fp64_oracle(n, ky, ty, ys):
    """The reverse step's column solves (Y^T wbar = lam) through the one-shot
    kernel (y_stage 2), the TMA-pipelined persistent clusters (y_stage 3) and
    the persistent CTAs whose column segments meet through global memory
    (y_stage 4) on grids with a partial last strip and partial chunks."""
    r = _window_parity(n, y_stage=ys, cols_per_cta=16, chunk_y=ky, cta_threads_y=ty)
    if r is None and ys == 4:
        pytest.skip("shape not supported by this staging mode")
    assert r is not None
    assert r < 1e-4, r


@pytest.mark.parametrize("n,kx", [(301, 16), (700, 32), (1000, 8), (129, 4)])
@pytest.mark.parametrize("xs", [2, 3])
def test_adjoint_row_solve_forms_match_fp64_oracle(n, kx, xs):
    """The reverse step's row solves and gradient terms with per-thread loads
    (x_stage 2) and with rows staged through shared memory (otherwise): odd
    and even row lengths, rows shorter than the padded row of the CTA, the
    source node inside a four-node group."""
    r = _window_parity(n, x_stage=xs, chunk_x=kx)
    if r is None:
        pytest.skip("shape not supported by this staging mode")
    assert r < 1e-4, r


def test_adjoint_taylor_start_and_initial_state():
    """Second-order start from a non-zero u(0): the start-up's dependence on m
    and f^0 is part of the gradient."""
    prob, m_true = inputs.adjoint_problem(48, 80, seed=2, n_rec=16)
    phi = 0.01 * inputs.standing_wave(48, 48)
    rng = np.random.default_rng(4)
    resid = f32(1e-3 * rng.standard_normal((80, 16)))
    hx = 1.0 / 49
    u0, u1 = oracle.adi_init(f32(prob.m).astype(np.float64), f32(phi).astype(np.float64), hx, hx,
                             prob.tau, taylor=True, wv0=float(f32(prob.wavelet)[0]), src=prob.src)
    ref = _oracle_grad(prob, prob.m, resid, u0, u1, start="taylor2")
    _, gm, gw = _gpu_grad(prob, 10, resid, phi=phi, start="taylor2")
    assert rel_l2(gm, ref["grad_m"]) < 1e-4
    assert rel_l2(gw, ref["grad_wavelet"]) < 1e-4


def test_adjoint_needs_checkpoints():
    import torch
    from paper_2006_10142_gb300 import api
    prob, _ = inputs.adjoint_problem(32, 10, seed=2, n_rec=16)
    dev = _dev()
    wav = torch.from_numpy(f32(prob.wavelet)).to(dev)
    h = api.AdiWave(torch.from_numpy(f32(prob.m)).to(dev), torch.zeros((32, 32), device=dev),
                    prob.tau, src=prob.src, wavelet=wav)
    tr = h.run(prob.steps, src=prob.src, wavelet=wav, rec=prob.rec)
    with pytest.raises(api.AdiError) as ei:
        h.adjoint(torch.zeros_like(tr))
    assert ei.value.code == 6
    h.close()


# ---------------------------------------------------------------------------
# the adjoint workload itself
# ---------------------------------------------------------------------------
@pytest.mark.slow
def test_adjoint_1024_full_run_matches_fp64_oracle():
    """adjoint_1024: 1024^2, 2000 steps, 64 receivers, checkpoint every 50,
    residual = oracle traces of m minus oracle data of the perturbed medium.
    The oracle keeps every forward field (about 17 GB of host memory)."""
    prob, m_true = inputs.adjoint_problem(1024, 2000, seed=0, n_rec=64)
    d = _oracle_traces(prob, m_true)
    tr_ref = _oracle_traces(prob, prob.m)
    resid = f32(tr_ref - d)
    tr, gm, gw = _gpu_grad(prob, 50, resid)
    assert rel_l2(tr, tr_ref) < 1e-4
    z = np.zeros((1024, 1024))
    ref = _oracle_grad(prob, prob.m, resid, z, z)
    e_m = rel_l2(gm, ref["grad_m"])
    e_w = rel_l2(gw, ref["grad_wavelet"])
    assert e_m < 1e-4 and e_w < 1e-4, (e_m, e_w)


@pytest.mark.slow
def test_adjoint_1024_finite_differences():
    """The adjoint workload: 1024^2, 2000 steps, 64 receivers, checkpoint every 50."""
    import torch
    from paper_2006_10142_gb300 import api
    prob, m_true = inputs.adjoint_problem(1024, 2000, seed=0, n_rec=64)
    dev = _dev()
    wav = torch.from_numpy(f32(prob.wavelet)).to(dev)
    zeros = torch.zeros((1024, 1024), device=dev)

    def traces(m):
        h = api.AdiWave(torch.from_numpy(f32(m)).to(dev), zeros, prob.tau, src=prob.src,
                        wavelet=wav)
        tr = h.run(prob.steps, src=prob.src, wavelet=wav, rec=prob.rec)
        h.sync_status()
        out = tr.double().cpu().numpy()
        h.close()
        return out

    d = traces(m_true)
    h = api.AdiWave(torch.from_numpy(f32(prob.m)).to(dev), zeros, prob.tau, src=prob.src,
                    wavelet=wav)
    h.set_checkpointing(50)
    tr = h.run(prob.steps, src=prob.src, wavelet=wav, rec=prob.rec)
    resid = tr.double().cpu().numpy() - d
    gm, _ = h.adjoint(torch.from_numpy(resid.astype(np.float32)).to(dev), ckpt_every=50)
    h.sync_status()
    g = gm.cpu().numpy()
    J = lambda t: 0.5 * np.sum((t - d) ** 2)
    errs = []
    for q in range(16):
        dm = inputs.smooth_direction(1024, q) * prob.m
        eps = 1e-3 * np.linalg.norm(prob.m) / np.linalg.norm(dm)
        fd = (J(traces(prob.m + eps * dm)) - J(traces(prob.m - eps * dm))) / (2 * eps)
        an = float(np.sum(g * dm))
        errs.append(abs(fd - an) / max(abs(fd), 1e-30))
    assert max(errs) < 1e-2, errs
    h.close()
