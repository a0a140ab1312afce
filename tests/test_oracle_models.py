"""Pins of the oracle's wider problem class and of the paper's literal
sub-schemes, against closed forms, scalar recurrences, dense solves and a
manufactured solution (no GPU).

- Eqs. (fr1)/(fr2) taken literally over half time levels (variant 1) and
  Listing 1's systems (variant 2): on the eigenmode sin(pi x) sin(pi y) with
  c = 1 and f = 0 every level is a multiple of the mode, and the 2D solves
  must reproduce the scalar recurrence of the mode's amplitude, whose
  closed form is known (variant 1: a rotation by theta per half level with
  cos theta = 1 / (1 + tau^2 P / 2); variant 2: damping by
  (1 + tau^2 P)^(-1/2) per half level).
- Eq. (CN1) with a time-dependent coefficient m^k = g_k m(x, y) and a source
  field: a manufactured solution converges at second order (a wrong sign
  or a dropped term of the time-dependent coefficient would leave first
  order); one step equals the dense factored solve.
"""
import math

import numpy as np
import pytest

import oracle


def _mode(nx, ny):
    x = (np.arange(nx) + 1.0) / (nx + 1)
    y = (np.arange(ny) + 1.0) / (ny + 1)
    return np.outer(np.sin(np.pi * y), np.sin(np.pi * x))


def _P(n):
    h = 1.0 / (n + 1)
    return 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2


@pytest.mark.parametrize("n,cfl,steps", [(31, 1.0, 40), (64, 0.5, 25), (127, 2.0, 10)])
def test_literal_subschemes_follow_the_mode_recurrence(n, cfl, steps):
    """Variant 1 from (u^{k-1/2}, u^k) = (phi, phi): the amplitudes of the
    half levels are a_q = cos((q - 1/2) theta) / cos(theta / 2)."""
    h = 1.0 / (n + 1)
    tau = cfl * h
    phi = _mode(n, n)
    a, b, _ = oracle.adi_run_halves(1, np.ones((n, n)), phi, phi, h, h, tau, steps)
    th = math.acos(1.0 / (1.0 + tau * tau * _P(n) / 2.0))
    amp = lambda q: math.cos((q - 0.5) * th) / math.cos(th / 2)
    np.testing.assert_allclose(a, amp(2 * steps) * phi, rtol=0, atol=1e-12)
    np.testing.assert_allclose(b, amp(2 * steps + 1) * phi, rtol=0, atol=1e-12)


@pytest.mark.parametrize("n,cfl,steps", [(31, 1.0, 40), (50, 0.3, 30)])
def test_listing1_systems_damp_the_mode_as_the_scalar_recurrence(n, cfl, steps):
    """Variant 2: (1 + tau^2 P) a_{q+1} = 2 a_q - a_{q-1}; the roots have
    modulus (1 + tau^2 P)^(-1/2)."""
    h = 1.0 / (n + 1)
    tau = cfl * h
    phi = _mode(n, n)
    a, b, _ = oracle.adi_run_halves(2, np.ones((n, n)), phi, phi, h, h, tau, steps)
    bq = 1.0 + tau * tau * _P(n)
    seq = [1.0, 1.0]
    for _ in range(2 * steps):
        seq.append((2.0 * seq[-1] - seq[-2]) / bq)
    np.testing.assert_allclose(a, seq[2 * steps] * phi, rtol=0, atol=1e-12)
    np.testing.assert_allclose(b, seq[2 * steps + 1] * phi, rtol=0, atol=1e-12)
    assert abs(seq[-1]) < bq ** (-0.5 * (2 * steps - 2)) * 2.0


def _lap1d(n, h):
    return (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) / h ** 2


def _dense_ops(nx, ny, hx, hy):
    Lx = np.kron(np.eye(ny), _lap1d(nx, hx))   # acts along rows (x fastest)
    Ly = np.kron(_lap1d(ny, hy), np.eye(nx))
    return Lx, Ly


@pytest.mark.parametrize("variant", [1, 2])
def test_half_level_step_equals_dense_solves(variant):
    """One step of each literal variant on a 7 x 5 grid with a variable
    coefficient and a point source, against numpy.linalg.solve of the two
    sub-problems written with dense operators."""
    nx, ny = 7, 5
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    tau = 0.7 * hx
    rng = np.random.default_rng(variant)
    m = 1.0 + rng.random((ny, nx))
    A = rng.standard_normal((ny, nx))
    B = rng.standard_normal((ny, nx))
    src, wk, wh = (2, 3), 0.8, -0.4
    uh, un = oracle.adi_step_halves(variant, m, A, B, hx, hy, tau, wk, wh, src)
    Lx, Ly = _dense_ops(nx, ny, hx, hy)
    M = np.diag(m.ravel())
    kfac = 0.5 * tau * tau if variant == 1 else tau * tau
    alpha = 1.0 if variant == 1 else 0.0
    S = 0.5 * tau * tau * M
    f = np.zeros(nx * ny)
    f[src[1] * nx + src[0]] = 1.0 / (hx * hy)
    r1 = 2 * B.ravel() - A.ravel() + alpha * S @ Lx @ A.ravel() + tau * tau * wk * f
    x1 = np.linalg.solve(np.eye(nx * ny) - kfac * M @ Lx, r1)
    r2 = 2 * x1 - B.ravel() + alpha * S @ Ly @ B.ravel() + tau * tau * wh * f
    x2 = np.linalg.solve(np.eye(nx * ny) - kfac * M @ Ly, r2)
    np.testing.assert_allclose(uh.ravel(), x1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(un.ravel(), x2, rtol=1e-12, atol=1e-12)


def test_time_dependent_step_equals_dense_factored_solve():
    """One step of Eq. (CN1) with m^k = g_k m and a source field against the
    dense factored system (I - S Lap_x)(I - S Lap_y) z = tau^2 (g_{k+1} m Lap u^k
    + (g_{k-1} - g_{k+1})/2 m Lap u^{k-1} + f^k) written out with numpy."""
    nx, ny = 6, 9
    hx, hy = 1.0 / (nx + 1), 1.0 / (ny + 1)
    tau = 0.9 * hy
    rng = np.random.default_rng(11)
    m = 1.0 + rng.random((ny, nx))
    up = rng.standard_normal((ny, nx))
    uc = rng.standard_normal((ny, nx))
    fk = rng.standard_normal((ny, nx))
    gp, gn = 0.8, 1.3
    un = oracle.adi_step_gen(m, up, uc, hx, hy, tau, gp, gn, fk, 0.5, (1, 4))
    Lx, Ly = _dense_ops(nx, ny, hx, hy)
    L = Lx + Ly
    M = np.diag(m.ravel())
    f = fk.ravel().copy()
    f[4 * nx + 1] += 0.5 / (hx * hy)
    r = tau * tau * (gn * M @ L @ uc.ravel() + 0.5 * (gp - gn) * M @ L @ up.ravel() + f)
    S = 0.5 * tau * tau * gn * M
    I = np.eye(nx * ny)
    z = np.linalg.solve((I - S @ Lx) @ (I - S @ Ly), r)
    np.testing.assert_allclose(un.ravel(), 2 * uc.ravel() - up.ravel() + z, rtol=1e-11, atol=1e-12)


def test_time_independent_case_reduces_to_the_plain_step():
    n = 20
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(3)
    m = 1.0 + rng.random((n, n))
    up, uc = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    a = oracle.adi_step(m, up, uc, h, h, 0.6 * h, wv=0.3, src=(4, 5))
    b = oracle.adi_step_gen(m, up, uc, h, h, 0.6 * h, 1.0, 1.0, None, 0.3, (4, 5))
    np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-14)


def _manufactured(n, T, omega=3.0):
    """u = sin(pi x) sin(2 pi y) cos(omega t) solves u_tt - g(t) m(x, y) Lap u = f
    with g(t) = 1 + 0.3 sin(2 t), m = 1 + 0.5 x y and
    f = (-omega^2 + 5 pi^2 g(t) m) u."""
    h = 1.0 / (n + 1)
    tau = h
    steps = int(round(T / tau))
    x = (np.arange(n) + 1.0) * h
    X, Y = np.meshgrid(x, x)
    m = 1.0 + 0.5 * X * Y
    shape = np.sin(np.pi * X) * np.sin(2 * np.pi * Y)
    g = 1.0 + 0.3 * np.sin(2.0 * tau * np.arange(steps + 3))
    f = np.array([(-omega ** 2 + 5 * np.pi ** 2 * g[k] * m) * shape * math.cos(omega * k * tau)
                  for k in range(steps + 2)])
    u0 = shape
    u1 = shape * math.cos(omega * tau)
    _, uc, _ = oracle.adi_run_gen(m, u0, u1, h, h, tau, steps, k0=1, g=g, f=f)
    exact = shape * math.cos(omega * (steps + 1) * tau)
    return float(np.max(np.abs(uc - exact)))


def test_time_dependent_coefficient_converges_at_second_order():
    errs = [_manufactured(n, 0.5) for n in (15, 31, 63)]
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert errs[-1] < 2e-3, errs
    assert all(3.3 < r < 4.8 for r in ratios), (errs, ratios)
