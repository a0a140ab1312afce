"""The seeded input recipes (no GPU): ranges, determinism and the fixed points
of the coefficient field, the Ricker wavelet, source and receiver placement
and the batch sizes, so that a change to a recipe cannot pass unnoticed."""
import math

import numpy as np
import pytest

from paper_2006_10142_gb300 import inputs


def test_grid_conventions():
    # Eq. f6: n interior nodes, h = l / (n + 1), x_i = (i + 1) h
    assert inputs.spacing(9) == pytest.approx(0.1)
    assert np.allclose(inputs.node_coords(4, 2.0), [0.4, 0.8, 1.2, 1.6])
    assert inputs.nearest_node(0.5, 9) == 4          # x_4 = 0.5
    assert inputs.nearest_node(-3.0, 9) == 0 and inputs.nearest_node(7.0, 9) == 8


def test_c_field_range_and_determinism():
    c = inputs.c_field(200, 150, seed=3)
    assert c.shape == (150, 200)
    assert c.min() > 1.0 and c.max() < 3.0            # 1 + 2 sigmoid(.)
    assert np.array_equal(c, inputs.c_field(200, 150, seed=3))
    assert not np.allclose(c, inputs.c_field(200, 150, seed=4))
    # row blocks only change how the sum is built
    assert np.array_equal(c, inputs.c_field(200, 150, seed=3, row_block=7))
    m = inputs.m_field(200, 150, seed=3)
    assert np.allclose(m, c * c)


def test_bump_draws_follow_the_recipe():
    p = inputs.draw_bumps(11)
    assert p.centres.shape == (8, 2) and p.widths.shape == (8,) and p.amps.shape == (8,)
    assert (p.centres >= 0).all() and (p.centres <= 1).all()
    assert (p.widths >= 0.05).all() and (p.widths <= 0.2).all()
    assert (np.abs(p.amps) <= 3).all()
    # the draw order is centres, widths, amplitudes from default_rng(seed)
    rng = np.random.default_rng(11)
    assert np.array_equal(p.centres, rng.uniform(0, 1, size=(8, 2)))
    assert np.array_equal(p.widths, rng.uniform(0.05, 0.2, size=8))
    assert np.array_equal(p.amps, rng.uniform(-3, 3, size=8))


def test_c_field_is_one_plus_two_sigmoid_of_the_bump_sum():
    nx, ny, seed = 17, 13, 5
    p = inputs.draw_bumps(seed)
    x, y = inputs.node_coords(nx), inputs.node_coords(ny)
    c = inputs.c_field(nx, ny, seed)
    for j, i in [(0, 0), (6, 9), (12, 16)]:
        s = sum(p.amps[b] * math.exp(-((x[i] - p.centres[b, 0]) ** 2 + (y[j] - p.centres[b, 1]) ** 2)
                                     / (2 * p.widths[b] ** 2)) for b in range(8))
        assert c[j, i] == pytest.approx(1 + 2 / (1 + math.exp(-s)), rel=1e-14)


def test_ricker_peak_and_zero_crossings():
    fp = inputs.RICKER_FP
    t0 = 1.0 / fp
    assert inputs.ricker(t0) == pytest.approx(1.0)
    # zeros where 2 pi^2 fp^2 (t - t0)^2 = 1; minima -2 exp(-3/2) at (t - t0)^2 = 3/(2 pi^2 fp^2)
    dz = 1.0 / (math.pi * fp * math.sqrt(2.0))
    assert abs(inputs.ricker(t0 + dz)) < 1e-14 and abs(inputs.ricker(t0 - dz)) < 1e-14
    dm = math.sqrt(1.5) / (math.pi * fp)
    assert inputs.ricker(t0 + dm) == pytest.approx(-2 * math.exp(-1.5))
    w = inputs.wavelet_samples(5, 0.01)
    assert np.allclose(w, inputs.ricker(np.arange(5) * 0.01))


def test_source_and_receivers():
    for seed in range(20):
        ix, iy = inputs.seeded_source(1000, seed)
        x, y = inputs.node_coords(1000)[[ix, iy]]
        assert 0.25 - 1e-3 <= x <= 0.75 + 1e-3 and 0.25 - 1e-3 <= y <= 0.75 + 1e-3
    rec = inputs.receiver_line(1024)
    assert rec.shape == (64, 2) and rec.dtype == np.int32
    assert (rec[:, 1] == inputs.nearest_node(0.1, 1024)).all()
    assert (np.diff(rec[:, 0]) > 0).all()
    xs = inputs.node_coords(1024)[rec[:, 0]]
    assert np.allclose(xs, (np.arange(64) + 0.5) / 64, atol=0.5 / 1025 + 1e-12)


def test_batch_sizes_and_problems():
    sizes = inputs.batch_sizes()
    assert len(sizes) == 64 and set(sizes) <= {256, 512, 1024, 2048}
    assert sizes == inputs.batch_sizes()
    prob = inputs.ricker_problem(64, 10, seed=2)
    c_max = math.sqrt(prob.m.max())
    assert prob.tau == pytest.approx(0.5 * inputs.spacing(64) / c_max)
    assert len(prob.wavelet) == 12 and not prob.phi.any()
    adj, m_true = inputs.adjoint_problem(64, 10, seed=0, n_rec=16)
    assert adj.src == (inputs.nearest_node(0.5, 64), inputs.nearest_node(0.9, 64))
    assert np.allclose(m_true, adj.m * (1 + 0.05 * inputs.bump(64, 64, 0.5, 0.5, 0.1)))
    assert adj.rec.shape == (16, 2)
