"""Seeded synthetic inputs for the 2D acoustic ADI workloads.

This module holds no arithmetic of the ADI method: it only draws and
evaluates the problem data (coefficient field, initial conditions, source
wavelet, source / receiver positions) that both the CUDA library and the FP64
oracle consume.  It imports neither of them, and nothing here depends on
torch or on a GPU.

Conventions (Section 2, Eq. f6): the unit square carries N = n + 1 intervals
per side, h = l / N, and the n interior nodes x_i = (i + 1) h, i = 0..n-1,
are the unknowns.  Arrays are row-major [ny][nx] with x fastest.

Recipes (the paper runs c = 1 with smooth data, Section 4; the larger
workloads add a heterogeneous medium and a point source):

- coefficient: c(x, y) = 1 + 2 sigmoid(sum_b A_b exp(-|p - p_b|^2 / (2 w_b^2)))
  with 8 bumps, centres p_b ~ U[0,1]^2, widths w_b ~ U[0.05, 0.2], amplitudes
  A_b ~ U[-3, 3], drawn from ``numpy.random.default_rng(seed)`` in that order;
  the scheme's coefficient is m = c^2.
- Ricker wavelet: w(t) = (1 - 2 pi^2 f^2 (t - t0)^2) exp(-pi^2 f^2 (t - t0)^2),
  peak frequency f = 20, t0 = 1 / f.
- point source: a node drawn uniformly in [0.25, 0.75]^2 (snapped to the
  nearest interior node), or a fixed position.
- receivers: 64 nodes at x_r = (r + 1/2) / 64 on the row nearest y = 0.1.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

N_BUMPS = 8
RICKER_FP = 20.0


def spacing(n: int, length: float = 1.0) -> float:
    """Grid step h = l / (n + 1) for n interior nodes (Eq. f6)."""
    return length / (n + 1)


def node_coords(n: int, length: float = 1.0) -> np.ndarray:
    """Interior node coordinates x_i = (i + 1) h, i = 0..n-1."""
    return (np.arange(n, dtype=np.float64) + 1.0) * spacing(n, length)


def nearest_node(x: float, n: int, length: float = 1.0) -> int:
    """Index of the interior node nearest to coordinate x (clamped)."""
    i = int(round(x / spacing(n, length))) - 1
    return min(max(i, 0), n - 1)


@dataclasses.dataclass(frozen=True)
class BumpParams:
    centres: np.ndarray   # [8, 2]
    widths: np.ndarray    # [8]
    amps: np.ndarray      # [8]


def draw_bumps(seed: int) -> BumpParams:
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(N_BUMPS, 2))
    widths = rng.uniform(0.05, 0.2, size=N_BUMPS)
    amps = rng.uniform(-3.0, 3.0, size=N_BUMPS)
    return BumpParams(centres, widths, amps)


def c_field(nx: int, ny: int, seed: int, lx: float = 1.0, ly: float = 1.0,
            dtype=np.float64, row_block: int = 1024) -> np.ndarray:
    """Speed c(x, y) = 1 + 2 sigmoid(sum of 8 seeded Gaussian bumps) in (1, 3).

    Each bump is separable, so the sum is built one block of rows at a time
    from outer products (FP64), then cast to ``dtype``.
    """
    p = draw_bumps(seed)
    x = node_coords(nx, lx)
    y = node_coords(ny, ly)
    gx = [np.exp(-(x - p.centres[b, 0]) ** 2 / (2.0 * p.widths[b] ** 2)) for b in range(N_BUMPS)]
    gy = [np.exp(-(y - p.centres[b, 1]) ** 2 / (2.0 * p.widths[b] ** 2)) for b in range(N_BUMPS)]
    out = np.empty((ny, nx), dtype=dtype)
    for j0 in range(0, ny, row_block):
        j1 = min(ny, j0 + row_block)
        s = np.zeros((j1 - j0, nx), dtype=np.float64)
        for b in range(N_BUMPS):
            s += p.amps[b] * np.outer(gy[b][j0:j1], gx[b])
        out[j0:j1] = 1.0 + 2.0 / (1.0 + np.exp(-s))
    return out


def m_field(nx: int, ny: int, seed: int, dtype=np.float64, **kw) -> np.ndarray:
    """Coefficient m = c^2 of the seeded c-field recipe."""
    c = c_field(nx, ny, seed, dtype=np.float64, **kw)
    return (c * c).astype(dtype)


def max_speed(nx: int, ny: int, seed: int) -> float:
    return float(c_field(nx, ny, seed).max())


def bump(nx: int, ny: int, cx: float, cy: float, width: float) -> np.ndarray:
    """Gaussian bump exp(-|p - (cx, cy)|^2 / (2 width^2)) on the interior nodes."""
    x = node_coords(nx)
    y = node_coords(ny)
    return np.outer(np.exp(-(y - cy) ** 2 / (2 * width ** 2)),
                    np.exp(-(x - cx) ** 2 / (2 * width ** 2)))


def standing_wave(nx: int, ny: int) -> np.ndarray:
    """phi = sin(pi x) sin(pi y) on the unit square's interior nodes."""
    return np.outer(np.sin(math.pi * node_coords(ny)), np.sin(math.pi * node_coords(nx)))


def ricker(t, fp: float = RICKER_FP, t0: Optional[float] = None):
    """Ricker wavelet (1 - 2 pi^2 fp^2 (t-t0)^2) exp(-pi^2 fp^2 (t-t0)^2)."""
    if t0 is None:
        t0 = 1.0 / fp
    a = (math.pi * fp * (np.asarray(t, dtype=np.float64) - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def wavelet_samples(n_levels: int, tau: float, fp: float = RICKER_FP) -> np.ndarray:
    """w(t_k) at t_k = k tau for k = 0..n_levels-1 (FP64)."""
    return ricker(np.arange(n_levels, dtype=np.float64) * tau, fp)


def seeded_source(n: int, seed: int) -> Tuple[int, int]:
    """Source node drawn uniformly in [0.25, 0.75]^2, snapped to the grid."""
    rng = np.random.default_rng(10_000 + seed)
    x, y = rng.uniform(0.25, 0.75, size=2)
    return nearest_node(x, n), nearest_node(y, n)


def receiver_line(n: int, count: int = 64, y: float = 0.1) -> np.ndarray:
    """[count, 2] int32 nodes at x_r = (r + 1/2)/count on the row nearest y."""
    iy = nearest_node(y, n)
    ix = [nearest_node((r + 0.5) / count, n) for r in range(count)]
    return np.array([[i, iy] for i in ix], dtype=np.int32)


def smooth_direction(n: int, seed: int, passes: int = 8) -> np.ndarray:
    """Seeded N(0,1) field smoothed by repeated 5-point averaging (FD directions)."""
    rng = np.random.default_rng(20_000 + seed)
    v = rng.standard_normal((n, n))
    for _ in range(passes):
        p = np.pad(v, 1)
        v = (p[1:-1, 1:-1] * 4 + p[:-2, 1:-1] + p[2:, 1:-1] + p[1:-1, :-2] + p[1:-1, 2:]) / 8.0
    return v


def batch_sizes(count: int = 64, seed: int = 0,
                choices: Sequence[int] = (256, 512, 1024, 2048)) -> List[int]:
    rng = np.random.default_rng(30_000 + seed)
    return [int(x) for x in rng.choice(np.asarray(choices), size=count)]


# ----------------------------------------------------------------------------
# The five workloads (names give what they are and their sizes).
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class GridProblem:
    """One grid: coefficient m (= c^2), initial state and point source."""
    n: int
    steps: int
    tau: float
    m: np.ndarray                      # [n, n] float64
    phi: np.ndarray                    # [n, n] float64
    psi: Optional[np.ndarray]          # [n, n] float64 or None (= 0)
    src: Optional[Tuple[int, int]]     # (ix, iy) or None
    wavelet: Optional[np.ndarray]      # w(t_k), k = 0..steps (float64) or None
    rec: Optional[np.ndarray] = None   # [n_rec, 2] int32


def standing_wave_problem(n: int = 128, steps: int = 200) -> GridProblem:
    """Unit square, c = 1, phi = sin(pi x) sin(pi y), psi = 0, no source, tau = h."""
    h = spacing(n)
    return GridProblem(n=n, steps=steps, tau=h, m=np.ones((n, n)), phi=standing_wave(n, n),
                       psi=None, src=None, wavelet=None)


def ricker_problem(n: int, steps: int, seed: int = 0, cfl: float = 0.5,
                   src: Optional[Tuple[int, int]] = None, with_wavelet: bool = True,
                   m_dtype=np.float64) -> GridProblem:
    """Seeded c-field, zero initial state, Ricker point source, tau = cfl h / max c."""
    m = m_field(n, n, seed, dtype=m_dtype)
    cmax = math.sqrt(float(m.max()))
    tau = cfl * spacing(n) / cmax
    if src is None:
        src = seeded_source(n, seed)
    wav = wavelet_samples(steps + 2, tau) if with_wavelet else None
    zeros = np.zeros((n, n), dtype=m_dtype)
    return GridProblem(n=n, steps=steps, tau=tau, m=m, phi=zeros, psi=None, src=src, wavelet=wav)


def adjoint_problem(n: int = 1024, steps: int = 2000, seed: int = 0,
                    n_rec: int = 64) -> Tuple[GridProblem, np.ndarray]:
    """Source at (0.5, 0.9), receivers along y = 0.1; returns (problem, m_true).

    The observed data come from the perturbed medium m_true = m (1 + 0.05 bump)
    with a bump of width 0.1 at (0.5, 0.5).
    """
    src = (nearest_node(0.5, n), nearest_node(0.9, n))
    prob = ricker_problem(n, steps, seed=seed, src=src)
    prob.rec = receiver_line(n, n_rec, 0.1)
    m_true = prob.m * (1.0 + 0.05 * bump(n, n, 0.5, 0.5, 0.1))
    return prob, m_true


WORKLOADS = {
    "standing_wave_128": dict(n=128, steps=200),
    "ricker_4096": dict(n=4096, steps=1000),
    "ricker_16384": dict(n=16384, steps=200),
    "batch_64_shots": dict(count=64, steps=500),
    "adjoint_1024": dict(n=1024, steps=2000, n_rec=64, ckpt_every=50),
}
