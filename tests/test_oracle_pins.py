"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-derive the oracle's own formula: each compares it with an
independent fact -- a dense library solve, an exact discrete closed form, the
continuous solution under mesh refinement, the unsplit scheme of Eq. (CN1),
a conserved discrete energy, a modal (discrete sine transform) solution of
the forced problem, and the paper's own Section 4 parameter set.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2006_10142_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------------------
# helpers (test-side, independent constructions)
# ---------------------------------------------------------------------------

def second_diff_matrix(n, h):
    """Dense 1D second difference with zero Dirichlet ends, / h^2."""
    return (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1)
            + np.diag(np.ones(n - 1), -1)) / (h * h)


def operators_2d(nx, ny, hx, hy):
    """Dense Lap_x, Lap_y acting on row-major [ny][nx] vectors (Kronecker form)."""
    Dx = second_diff_matrix(nx, hx)
    Dy = second_diff_matrix(ny, hy)
    Lx = np.kron(np.eye(ny), Dx)
    Ly = np.kron(Dy, np.eye(nx))
    return Lx, Ly


def mode_eig(p, n, h):
    """-Lap_1D sin(p pi x) = P sin(p pi x),  P = 4/h^2 sin^2(p pi h / 2)."""
    return 4.0 / (h * h) * math.sin(p * math.pi * h / 2.0) ** 2


def sine_mode(nx, ny, p, q):
    x = inputs.node_coords(nx)
    y = inputs.node_coords(ny)
    return np.outer(np.sin(q * math.pi * y), np.sin(p * math.pi * x))


# ---------------------------------------------------------------------------
# P-dense: tridiagonal solves and one full step vs dense linear algebra
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 33])
def test_thomas_matches_dense_solve(oracle_mod, n):
    rng = np.random.default_rng(n)
    a = rng.uniform(-1, 1, n)
    c = rng.uniform(-1, 1, n)
    b = np.abs(a) + np.abs(c) + rng.uniform(0.1, 2.0, n)
    b *= rng.choice([-1.0, 1.0], n)
    d = rng.standard_normal(n)
    A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    x_ref = np.linalg.solve(A, d)
    x = oracle_mod.thomas(a, b, c, d)
    np.testing.assert_allclose(x, x_ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("nx,ny", [(7, 5), (6, 9), (12, 12)])
def test_step_matches_dense_factored_solve(oracle_mod, nx, ny):
    """u^{k+1} = 2u^k - u^{k-1} + z with (I - S Lx)(I - S Ly) z = tau^2 (m Lap u^k + f)."""
    rng = np.random.default_rng(nx * 100 + ny)
    hx, hy = oracle_mod.grid_steps(nx, ny)
    tau = 0.7 * min(hx, hy)
    m = rng.uniform(1.0, 9.0, (ny, nx))
    up = rng.standard_normal((ny, nx))
    uc = rng.standard_normal((ny, nx))
    src = (nx // 2, ny // 3)
    wv = 0.37
    Lx, Ly = operators_2d(nx, ny, hx, hy)
    S = np.diag(tau * tau * m.ravel() / 2.0)
    N = nx * ny
    X = np.eye(N) - S @ Lx
    Y = np.eye(N) - S @ Ly
    f = np.zeros(N)
    f[src[1] * nx + src[0]] = wv / (hx * hy)
    r = tau * tau * (m.ravel() * ((Lx + Ly) @ uc.ravel()) + f)
    z = np.linalg.solve(X @ Y, r)
    ref = (2 * uc.ravel() - up.ravel() + z).reshape(ny, nx)
    got, r_o, w_o, z_o = oracle_mod.adi_step(m, up, uc, hx, hy, tau, wv=wv, src=src,
                                             return_parts=True)
    np.testing.assert_allclose(r_o.ravel(), r, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(w_o.ravel(), np.linalg.solve(X, r), rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(got, ref, rtol=1e-11, atol=1e-11)


# ---------------------------------------------------------------------------
# P-exact: the discrete closed form of the standing wave
# ---------------------------------------------------------------------------

def exact_mode_amplitude(K, nx, ny, tau, m, v1):
    """Scalar recurrence of the (1,1) eigenmode under the factored scheme.

    (1 + s Px)(1 + s Py) (v^{k+1} - 2 v^k + v^{k-1}) = -tau^2 m (Px + Py) v^k,
    s = tau^2 m / 2, so v^k = cos(k th) + B sin(k th) with
    cos th = 1 - tau^2 m (Px + Py) / (2 (1 + s Px)(1 + s Py)), v^0 = 1, v^1 = v1.
    """
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    Px, Py = mode_eig(1, nx, hx), mode_eig(1, ny, hy)
    s = tau * tau * m / 2.0
    cos_th = 1.0 - tau * tau * m * (Px + Py) / (2.0 * (1 + s * Px) * (1 + s * Py))
    th = math.acos(cos_th)
    B = (v1 - math.cos(th)) / math.sin(th)
    return math.cos(K * th) + B * math.sin(K * th)


@pytest.mark.parametrize("nx,ny,m,steps", [(128, 128, 1.0, 200), (40, 24, 2.5, 90)])
def test_standing_wave_exact_discrete_solution(oracle_mod, nx, ny, m, steps):
    hx, hy = oracle_mod.grid_steps(nx, ny)
    tau = min(hx, hy)
    phi = inputs.standing_wave(nx, ny)
    M = np.full((ny, nx), m)
    u0, u1 = oracle_mod.adi_init(M, phi, hx, hy, tau)
    _, uK, _ = oracle_mod.adi_run(M, u0, u1, hx, hy, tau, steps)
    amp = exact_mode_amplitude(steps + 1, nx, ny, tau, m, 1.0)
    # paper start (v^1 = 1) reduces to cos((K - 1/2) th) / cos(th / 2)
    err = np.abs(uK - amp * phi).max()
    assert err < 1e-11, err


def test_standing_wave_with_velocity_and_taylor_start(oracle_mod):
    nx = ny = 48
    hx, hy = oracle_mod.grid_steps(nx, ny)
    tau = 0.8 * hx
    m = 1.7
    M = np.full((ny, nx), m)
    phi = inputs.standing_wave(nx, ny)
    beta = 0.6
    u0, u1 = oracle_mod.adi_init(M, phi, hx, hy, tau, psi=beta * phi, taylor=True)
    # u^1 = phi + tau psi + tau^2/2 m Lap phi; Lap phi = -(Px + Py) phi
    Px, Py = mode_eig(1, nx, hx), mode_eig(1, ny, hy)
    v1 = 1.0 + tau * beta - 0.5 * tau * tau * m * (Px + Py)
    np.testing.assert_allclose(u1, v1 * phi, rtol=0, atol=1e-13)
    _, uK, _ = oracle_mod.adi_run(M, u0, u1, hx, hy, tau, 75)
    amp = exact_mode_amplitude(76, nx, ny, tau, m, v1)
    assert np.abs(uK - amp * phi).max() < 1e-11


def test_paper_section4_parameters(oracle_mod):
    """The paper's own run (Section 4): dx = 0.01, c = 1, dt = 0.02, T = 1, 50 steps."""
    with open(os.path.join(HERE, "golden", "paper_section4_experiment.json")) as f:
        g = json.load(f)
    n = int(round(1.0 / g["dx"])) - 1
    assert n == 99
    tau = g["dt"]
    levels = int(round(g["T"] / tau))
    assert levels == g["time_steps"]
    hx, hy = oracle_mod.grid_steps(n, n)
    phi = inputs.standing_wave(n, n)
    M = np.full((n, n), g["c"] ** 2)
    u0, u1 = oracle_mod.adi_init(M, phi, hx, hy, tau)
    _, u_T, _ = oracle_mod.adi_run(M, u0, u1, hx, hy, tau, levels - 1)
    amp = exact_mode_amplitude(levels, n, n, tau, g["c"] ** 2, 1.0)
    assert np.abs(u_T - amp * phi).max() < 1e-11
    # tau = 2h: the implicit scheme stays bounded (unconditional stability)
    assert np.abs(u_T).max() <= 1.0 + 1e-12


# ---------------------------------------------------------------------------
# P-cont: convergence to the continuous standing wave
# ---------------------------------------------------------------------------

def cont_error(oracle_mod, n, taylor):
    h = 1.0 / (n + 1)
    tau = h
    T = 1.5
    steps = int(round(T / tau)) - 1
    phi = inputs.standing_wave(n, n)
    M = np.ones((n, n))
    u0, u1 = oracle_mod.adi_init(M, phi, h, h, tau, taylor=taylor)
    _, uT, _ = oracle_mod.adi_run(M, u0, u1, h, h, tau, steps)
    t = (steps + 1) * tau
    exact = phi * math.cos(math.sqrt(2.0) * math.pi * t)
    return np.linalg.norm(uT - exact) / np.linalg.norm(phi)


def test_mesh_refinement_orders(oracle_mod):
    ns = [31, 63, 127]
    e_paper = [cont_error(oracle_mod, n, False) for n in ns]
    e_taylor = [cont_error(oracle_mod, n, True) for n in ns]
    r_paper = [e_paper[i] / e_paper[i + 1] for i in range(2)]
    r_taylor = [e_taylor[i] / e_taylor[i + 1] for i in range(2)]
    # Eq. (CN2)'s first-order start: the overall error is O(tau + h^2)
    assert all(1.7 < r < 2.4 for r in r_paper), (e_paper, r_paper)
    # second-order start: the scheme's own O(tau^2 + h^2)
    assert all(3.4 < r < 4.6 for r in r_taylor), (e_taylor, r_taylor)
    assert e_taylor[-1] < 5e-3


# ---------------------------------------------------------------------------
# P-CN: the factored step differs from the unsplit Eq. (CN1) solve by O(tau^4) relative to z
# ---------------------------------------------------------------------------

def test_factored_vs_unsplit_cn1(oracle_mod):
    nx = ny = 15
    hx, hy = oracle_mod.grid_steps(nx, ny)
    x = inputs.node_coords(nx)
    m = 1.0 + 0.5 * np.outer(np.cos(2 * x), np.sin(3 * x))
    up = np.outer(np.sin(math.pi * x), np.sin(2 * math.pi * x))
    uc = 0.9 * up
    Lx, Ly = operators_2d(nx, ny, hx, hy)
    diffs = []
    for tau in (0.2 * hx, 0.1 * hx):
        got = oracle_mod.adi_step(m, up, uc, hx, hy, tau)
        # Eq. (CN1): (u+ - 2u + u-)/tau^2 - m/2 Lap u+ - m/2 Lap u- = 0, solved densely
        A = np.eye(nx * ny) / tau ** 2 - 0.5 * np.diag(m.ravel()) @ (Lx + Ly)
        rhs = (2 * uc.ravel() - up.ravel()) / tau ** 2 + 0.5 * m.ravel() * ((Lx + Ly) @ up.ravel())
        cn = np.linalg.solve(A, rhs).reshape(ny, nx)
        z = cn - 2 * uc + up
        # the splitting term s^2 Lap_x Lap_y z is O(tau^4) relative to z
        diffs.append(np.abs(got - cn).max() / np.abs(z).max())
    ratio = diffs[0] / diffs[1]
    assert 12.0 < ratio < 20.0, (diffs, ratio)


# ---------------------------------------------------------------------------
# P-energy: conserved discrete energy on a homogeneous medium
# ---------------------------------------------------------------------------

def _lap1(u, axis, h):
    p = np.pad(u, 1)
    if axis == 1:
        return (p[1:-1, :-2] - 2 * u + p[1:-1, 2:]) / h ** 2
    return (p[:-2, 1:-1] - 2 * u + p[2:, 1:-1]) / h ** 2


def energy(u_new, u_old, tau, m, hx, hy):
    v = (u_new - u_old) / tau
    w = 0.5 * (u_new + u_old)
    s = tau * tau * m / 2.0
    lap = lambda a: _lap1(a, 1, hx) + _lap1(a, 0, hy)
    return (np.sum(v * v) + tau * tau * m / 4.0 * np.sum(-lap(v) * v)
            + s * s * np.sum(_lap1(_lap1(v, 0, hy), 1, hx) * v) + m * np.sum(-lap(w) * w))


def test_energy_conservation_homogeneous(oracle_mod):
    nx, ny = 20, 26
    hx, hy = oracle_mod.grid_steps(nx, ny)
    tau = 1.5 * hx
    m = 2.0
    rng = np.random.default_rng(3)
    up = rng.standard_normal((ny, nx))
    uc = up + 0.1 * rng.standard_normal((ny, nx))
    M = np.full((ny, nx), m)
    e0 = energy(uc, up, tau, m, hx, hy)
    es = []
    for _ in range(40):
        un = oracle_mod.adi_step(M, up, uc, hx, hy, tau)
        up, uc = uc, un
        es.append(energy(uc, up, tau, m, hx, hy))
    drift = max(abs(e - e0) for e in es) / e0
    assert drift < 1e-12, drift


# ---------------------------------------------------------------------------
# P-modal: a point source projected on the discrete sine modes
# ---------------------------------------------------------------------------

def test_point_source_modal_solution(oracle_mod):
    """Constant m: each sine mode (p, q) obeys its own forced scalar recurrence

    (1 + s Pp)(1 + s Pq)(v^{k+1} - 2v^k + v^{k-1}) = tau^2 (-m (Pp + Pq) v^k + g^k),
    g^k = 4 w(t_k) sin(p pi x_a) sin(q pi y_b) -- the discrete sine coefficient of
    the point source w(t_k) / (h1 h2) at node (a, b).
    """
    nx, ny = 13, 9
    hx, hy = oracle_mod.grid_steps(nx, ny)
    tau = 0.9 * hx
    m = 1.3
    M = np.full((ny, nx), m)
    src = (4, 6)
    steps = 30
    wav = np.sin(0.3 * np.arange(steps + 2)) * np.exp(-0.05 * np.arange(steps + 2))
    z = np.zeros((ny, nx))
    _, _, traces = oracle_mod.adi_run(M, z, z, hx, hy, tau, steps, k0=1, src=src, wavelet=wav,
                                      rec=np.array([[x, y] for y in range(ny) for x in range(nx)]))
    x = inputs.node_coords(nx)
    y = inputs.node_coords(ny)
    s = tau * tau * m / 2.0
    for (p, q) in [(1, 1), (2, 3), (5, 2), (13, 9)]:
        Pp, Pq = mode_eig(p, nx, hx), mode_eig(q, ny, hy)
        den = (1 + s * Pp) * (1 + s * Pq)
        amp = 4.0 * math.sin(p * math.pi * x[src[0]]) * math.sin(q * math.pi * y[src[1]])
        vm, vc = 0.0, 0.0
        mode = sine_mode(nx, ny, p, q)
        for k in range(steps):
            level = 1 + k
            vn = 2 * vc - vm + tau * tau * (-m * (Pp + Pq) * vc + amp * wav[level]) / den
            vm, vc = vc, vn
            field = traces[k].reshape(ny, nx)
            coef = (2.0 / (nx + 1)) * (2.0 / (ny + 1)) * np.sum(field * mode)
            assert abs(coef - vn) < 1e-11 * max(1.0, abs(vn)), (p, q, k, coef, vn)
