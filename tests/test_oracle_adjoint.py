"""Pins of the oracle's reverse-mode gradient against central finite differences.

The forward run is itself pinned (test_oracle_pins.py); the misfit
J = 1/2 sum_s sum_r (u^{k0+s+1}(rec r) - d_{s,r})^2 is differentiated through it
numerically, in FP64, along seeded directions.  A wrong sign, a transposed
sweep taken in the wrong order or a missing gradient term fails these.
"""
import numpy as np
import pytest

from paper_2006_10142_gb300 import inputs


def _setup(nx=18, ny=14, steps=36, seed=1):
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    m = inputs.m_field(nx, ny, seed)
    tau = 0.5 * min(hx, hy) / np.sqrt(m.max()) * 3.0
    src = (nx // 2, ny - 3)
    wav = inputs.ricker(np.arange(steps + 2) * tau, fp=4.0, t0=0.05)
    rec = np.array([[i, 2] for i in range(1, nx - 1, 3)], dtype=np.int32)
    rng = np.random.default_rng(seed)
    u_prev = 0.01 * rng.standard_normal((ny, nx))
    u_cur = u_prev + 0.001 * rng.standard_normal((ny, nx))
    return dict(nx=nx, ny=ny, hx=hx, hy=hy, tau=tau, m=m, src=src, wav=wav, rec=rec,
                steps=steps, u_prev=u_prev, u_cur=u_cur)


def _misfit(oracle_mod, P, m, wav, d, taylor=False):
    if taylor:
        u0, u1 = oracle_mod.adi_init(m, P["u_prev"], P["hx"], P["hy"], P["tau"], taylor=True,
                                     wv0=wav[0], src=P["src"])
    else:
        u0, u1 = P["u_prev"], P["u_cur"]
    _, _, tr = oracle_mod.adi_run(m, u0, u1, P["hx"], P["hy"], P["tau"], P["steps"], k0=1,
                                  src=P["src"], wavelet=wav, rec=P["rec"])
    return 0.5 * np.sum((tr - d) ** 2), tr, (u0, u1)


@pytest.mark.parametrize("taylor", [False, True])
def test_adjoint_gradient_matches_central_differences(oracle_mod, taylor):
    P = _setup()
    m_true = P["m"] * (1.0 + 0.05 * inputs.bump(P["nx"], P["ny"], 0.5, 0.5, 0.15))
    _, d, _ = _misfit(oracle_mod, P, m_true, P["wav"], 0.0, taylor)
    J0, tr, (u0, u1) = _misfit(oracle_mod, P, P["m"], P["wav"], d, taylor)
    g = oracle_mod.adi_adjoint(P["m"], u0, u1, P["hx"], P["hy"], P["tau"], P["steps"], tr - d,
                               P["rec"], k0=1, src=P["src"], wavelet=P["wav"], taylor_k0=taylor)
    rng = np.random.default_rng(7)
    for trial in range(4):
        dm = rng.standard_normal(P["m"].shape)
        eps = 1e-6 * np.linalg.norm(P["m"]) / np.linalg.norm(dm)
        Jp, _, _ = _misfit(oracle_mod, P, P["m"] + eps * dm, P["wav"], d, taylor)
        Jm, _, _ = _misfit(oracle_mod, P, P["m"] - eps * dm, P["wav"], d, taylor)
        fd = (Jp - Jm) / (2 * eps)
        an = np.sum(g["grad_m"] * dm)
        assert abs(fd - an) <= 1e-6 * abs(fd) + 1e-14, (trial, fd, an)
    # wavelet gradient
    for trial in range(2):
        dw = rng.standard_normal(P["wav"].shape)
        eps = 1e-6 * np.linalg.norm(P["wav"]) / np.linalg.norm(dw)
        Jp, _, _ = _misfit(oracle_mod, P, P["m"], P["wav"] + eps * dw, d, taylor)
        Jm, _, _ = _misfit(oracle_mod, P, P["m"], P["wav"] - eps * dw, d, taylor)
        fd = (Jp - Jm) / (2 * eps)
        an = np.sum(g["grad_wavelet"] * dw)
        assert abs(fd - an) <= 1e-6 * abs(fd) + 1e-14, (trial, fd, an)


def test_adjoint_state_gradients(oracle_mod):
    """dJ/du^{k0} and dJ/du^{k0-1} (the adjoint fields left after the reverse sweep)."""
    P = _setup(nx=12, ny=10, steps=20)
    rng = np.random.default_rng(11)
    d = rng.standard_normal((P["steps"], P["rec"].shape[0])) * 1e-3
    _, _, tr = oracle_mod.adi_run(P["m"], P["u_prev"], P["u_cur"], P["hx"], P["hy"], P["tau"],
                                  P["steps"], src=P["src"], wavelet=P["wav"], rec=P["rec"])
    g = oracle_mod.adi_adjoint(P["m"], P["u_prev"], P["u_cur"], P["hx"], P["hy"], P["tau"],
                               P["steps"], tr - d, P["rec"], src=P["src"], wavelet=P["wav"])

    def J(up, uc):
        _, _, t = oracle_mod.adi_run(P["m"], up, uc, P["hx"], P["hy"], P["tau"], P["steps"],
                                     src=P["src"], wavelet=P["wav"], rec=P["rec"])
        return 0.5 * np.sum((t - d) ** 2)

    du = rng.standard_normal(P["u_cur"].shape)
    eps = 1e-5
    fd_c = (J(P["u_prev"], P["u_cur"] + eps * du) - J(P["u_prev"], P["u_cur"] - eps * du)) / (2 * eps)
    fd_p = (J(P["u_prev"] + eps * du, P["u_cur"]) - J(P["u_prev"] - eps * du, P["u_cur"])) / (2 * eps)
    assert abs(fd_c - np.sum(g["lam_cur"] * du)) <= 1e-6 * abs(fd_c)
    assert abs(fd_p - np.sum(g["lam_prev"] * du)) <= 1e-6 * abs(fd_p)


def _dense_lap_1d(n, h):
    """Second difference with the zero Dirichlet ring, as an n x n matrix."""
    return (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1)
            + np.diag(np.ones(n - 1), -1)) / (h * h)


@pytest.mark.parametrize("nx,ny", [(9, 7), (1, 5), (12, 1)])
def test_single_sweeps_and_transposes_match_dense_solves(oracle_mod, nx, ny):
    """X = I - S Lap_x and Y = I - S Lap_y (S = diag(tau^2 m / 2)) and their
    transposes, built as dense matrices over the whole grid and solved by
    numpy.linalg.solve, against the oracle's sweeps; then the dot-product
    identity <Op^{-T} a, b> = <a, Op^{-1} b> for each operator."""
    rng = np.random.default_rng(nx * 31 + ny)
    hx, hy, tau = 1.0 / (nx + 1), 0.7 / (ny + 1), 0.03
    m = 1.0 + 3.0 * rng.random((ny, nx))
    S = np.diag(tau * tau * m.ravel() / 2.0)   # unknowns ordered j * nx + i
    Lx = np.kron(np.eye(ny), _dense_lap_1d(nx, hx))
    Ly = np.kron(_dense_lap_1d(ny, hy), np.eye(nx))
    ops = {1: (np.eye(nx * ny) - S @ Lx, hx), 0: (np.eye(nx * ny) - S @ Ly, hy)}
    a = rng.standard_normal((ny, nx))
    b = rng.standard_normal((ny, nx))
    for axis, (A, h) in ops.items():
        fwd = oracle_mod.line_sweep(m, b, h, tau, axis)
        tr = oracle_mod.line_sweep(m, a, h, tau, axis, transposed=True)
        assert np.allclose(fwd.ravel(), np.linalg.solve(A, b.ravel()), rtol=1e-12, atol=1e-13)
        assert np.allclose(tr.ravel(), np.linalg.solve(A.T, a.ravel()), rtol=1e-12, atol=1e-13)
        lhs, rhs = np.vdot(tr, b), np.vdot(a, fwd)
        assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))


def test_transposed_stencil_of_the_right_hand_side(oracle_mod):
    """The reverse step takes tau^2 Lap(m . rbar) for the transpose of
    u -> tau^2 m . Lap u: <m . Lap u, v> = <u, Lap(m . v)> (Lap symmetric with
    the zero Dirichlet ring), on a non-square grid with h1 != h2."""
    rng = np.random.default_rng(3)
    ny, nx = 11, 16
    hx, hy = 1.0 / (nx + 1), 1.3 / (ny + 1)
    m = 1.0 + rng.random((ny, nx))
    u = rng.standard_normal((ny, nx))
    v = rng.standard_normal((ny, nx))
    lhs = np.vdot(m * oracle_mod.laplacian(u, hx, hy), v)
    rhs = np.vdot(u, oracle_mod.laplacian(m * v, hx, hy))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs))
