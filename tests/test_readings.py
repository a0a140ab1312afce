"""Executable evidence for reading C3: the paper's two sub-problems (Eqs. fr1,
fr2) taken literally do not advance the wave at its speed, while the
factored delta-form of Eq. CN1 that this library solves does.

For the eigenmode sin(pi x) sin(pi y) of the discrete Laplacian (each of
Lap_x, Lap_y has eigenvalue -P, P = (4/h^2) sin^2(pi h/2)), c = 1 and f = 0,
both schemes reduce to scalar recurrences:

- Eqs. fr1 / fr2 alternate over the levels k - 1/2, k, k + 1/2, k + 1, ...;
  each is a three-level relation with a full tau^2 and half of one
  direction's operator at its outer levels:
  (w_{n+1} - 2 w_n + w_{n-1}) / tau^2 + (P / 2)(w_{n+1} + w_{n-1}) = 0,
  so cos(theta_half) = 1 / (1 + tau^2 P / 2) per half level;
- the factored delta-form (I - S Lap_x)(I - S Lap_y) z = tau^2 Lap u^k with
  S = tau^2 / 2 gives (1 + S P)^2 (v^{k+1} - 2 v^k + v^{k-1}) = -2 tau^2 P v^k,
  so cos(theta) = 1 - tau^2 P / (1 + S P)^2 per step;
- the semi-discrete wave v'' = -2 P v turns by tau sqrt(2 P) per step.
"""
import math

import numpy as np
import pytest


def _phases(n, cfl):
    h = 1.0 / (n + 1)
    tau = cfl * h
    P = 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    literal = 2.0 * math.acos(1.0 / (1.0 + tau * tau * P / 2.0))   # two half levels per step
    S = tau * tau / 2.0
    factored = math.acos(1.0 - tau * tau * P / (1.0 + S * P) ** 2)
    exact = tau * math.sqrt(2.0 * P)
    return literal, factored, exact


@pytest.mark.parametrize("n,cfl", [(128, 1.0), (512, 1.0), (512, 0.25), (2048, 0.5)])
def test_literal_subschemes_run_about_sqrt2_too_fast(n, cfl):
    literal, factored, exact = _phases(n, cfl)
    assert literal / exact == pytest.approx(math.sqrt(2.0), rel=2e-3)
    assert factored / exact == pytest.approx(1.0, rel=2e-3)


def test_literal_recurrence_iterated_matches_its_closed_form():
    # iterate the alternating half-level recurrence itself and compare the
    # phase it accumulates with the closed form used above
    n, cfl, steps = 128, 1.0, 60
    h = 1.0 / (n + 1)
    tau = cfl * h
    P = 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    a = 1.0 + tau * tau * P / 2.0
    th = math.acos(1.0 / a)
    w = [1.0, math.cos(th)]                    # a pure cosine start
    for _ in range(2 * steps - 1):
        w.append(2.0 * w[-1] / a - w[-2])
    expect = [math.cos(k * th) for k in range(len(w))]
    assert np.allclose(w, expect, atol=1e-10)
    literal, _, exact = _phases(n, cfl)
    # after `steps` full steps the literal scheme is far out of phase with the wave
    assert abs(math.cos(steps * literal) - math.cos(steps * exact)) > 0.5


def test_listing1_coefficients_damp_every_mode():
    """Reading C4: Listing 1's a = c = tau^2, b = 2 tau^2 + h^2,
    f = h^2 u_old - 2 h^2 u^k, in the convention a y_{i-1} - b y_i + c y_{i+1} = f,
    is the fully implicit (y - 2 u^k + u_old) / tau^2 = Lap_x y.  On one mode
    its two roots have |r|^2 = 1 / (1 + tau^2 P) < 1 (every mode decays), while
    the factored delta-form's roots lie on the unit circle (no damping)."""
    n, cfl = 128, 1.0
    h = 1.0 / (n + 1)
    tau = cfl * h
    P = 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    # the listing's row equation applied to the mode sin(pi x): y_{i-1} + y_{i+1} = (2 - h^2 P) y_i
    a = c = tau * tau
    b = 2 * tau * tau + h * h
    lhs = a * (2 - h * h * P) - b            # coefficient of y_i after the neighbours
    # lhs * y = h^2 (u_old - 2 u^k)  <=>  (1 + tau^2 P) y - 2 u^k + u_old = 0
    assert -lhs / (h * h) == pytest.approx(1 + tau * tau * P, rel=1e-12)
    r_listing = np.roots([1 + tau * tau * P, -2.0, 1.0])
    assert np.allclose(np.abs(r_listing), (1 + tau * tau * P) ** -0.5)
    assert (np.abs(r_listing) < 1).all()
    S = tau * tau / 2
    q = (1 + S * P) ** 2
    r_factored = np.roots([q, -(2 * q - 2 * tau * tau * P), q])
    assert np.allclose(np.abs(r_factored), 1.0)
    # iterating the listing's recurrence: the amplitude decays as |r|^n
    w = [1.0, 1.0]
    for _ in range(200):
        w.append((2 * w[-1] - w[-2]) / (1 + tau * tau * P))
    env = (1 + tau * tau * P) ** -0.5
    assert max(abs(x) for x in w[-20:]) < 2 * env ** 180
