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
