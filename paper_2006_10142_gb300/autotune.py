"""Autotuner for the line-solver launch parameters of one grid shape.

Knobs (see ``adi_wave_tuning`` in include/adiwave.h): systems (rows) per CTA
of the x sweep, unknowns per thread in each sweep, strip width of the y sweep,
threads per CTA, the interface solver (warp-shuffle block CR + PCR, or
shared-memory CR handing `pcr_size` equations to warp PCR -- the CR-to-PCR
switch level) and graph replay.

Each candidate runs a few steps of a c = 1 problem of the requested shape
(the kernels do the same work for any coefficient) with per-kernel CUDA
events on the launching stream.  The x-sweep and y-sweep knobs act on
different kernels, so every timed run contributes one x candidate and one y
candidate; the shared knobs (solver, threads per CTA) are searched around
them.  Results are cached per (device, nx, ny, precision) in a JSON file
(``$ADIWAVE_TUNE_CACHE`` or ``~/.cache/adiwave/tuning.json``).
"""
from __future__ import annotations

import itertools
import json
import math
import os
from typing import Dict, List, Optional

X_KNOBS = ("chunk_x", "rows_per_cta", "cta_threads")
Y_KNOBS = ("chunk_y", "cols_per_cta", "cta_threads_y", "y_stage")
SHARED_KNOBS = ("solver", "pcr_size")


def cache_path() -> str:
    return os.environ.get("ADIWAVE_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "adiwave", "tuning.json"))


def _key(device_name: str, nx: int, ny: int, fp64: str) -> str:
    return "%s|%dx%d|%s" % (device_name, nx, ny, fp64)


def _load_cache() -> Dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(data: Dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp.%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def candidates(nx: int, ny: int):
    """(shared settings, x candidates, y candidates) for a grid shape."""
    shared = [dict(solver=1, pcr_size=0), dict(solver=2, pcr_size=8), dict(solver=2, pcr_size=32)]
    xs = [dict(chunk_x=k, rows_per_cta=0, cta_threads=t)
          for k, t in itertools.product((8, 16, 32), (256, 512, 1024))]
    ys = [dict(chunk_y=k, cols_per_cta=w, cta_threads_y=t, y_stage=s)
          for k, w, t, s in itertools.product((8, 16, 32), (8, 16), (256, 512, 1024), (1, 2))]
    return shared, xs, ys


def tune(nx: int, ny: int, fp64: str = "auto", steps: int = 3, warmup: int = 1,
         use_cache: bool = True, verbose: bool = False) -> Dict:
    """Best tuning for an nx x ny grid: {'tuning': {...}, 'x_ms': .., 'y_ms': ..}."""
    import numpy as np
    import torch

    from . import api

    dev = torch.device("cuda", torch.cuda.current_device())
    name = torch.cuda.get_device_name(dev)
    key = _key(name, nx, ny, fp64)
    cache = _load_cache() if use_cache else {}
    if key in cache:
        return cache[key]

    m = torch.ones((ny, nx), dtype=torch.float32, device=dev)
    h = min(1.0 / (nx + 1), 1.0 / (ny + 1))
    tau = 0.5 * h
    sim = api.AdiWave(m, torch.zeros_like(m), tau, fp64=fp64)
    shared, xs, ys = candidates(nx, ny)
    best_x: Dict[int, tuple] = {}
    best_y: Dict[int, tuple] = {}
    n = max(len(xs), len(ys))
    for si, sh in enumerate(shared):
        for i in range(n):
            cfg = dict(sh)
            cfg.update(xs[i % len(xs)])
            cfg.update(ys[i % len(ys)])
            try:
                sim.set_tuning(**cfg)
            except api.AdiError:
                continue
            sim.run(warmup)
            sim.profile(True)
            sim.profile_read()
            sim.run(steps)
            ms, cnt = sim.profile_read()
            sim.profile(False)
            x_ms, y_ms = ms[0] / max(cnt[0], 1), ms[1] / max(cnt[1], 1)
            if verbose:
                print(json.dumps({"cfg": cfg, "x_ms": x_ms, "y_ms": y_ms}))
            if si not in best_x or x_ms < best_x[si][0]:
                best_x[si] = (x_ms, {k: cfg[k] for k in X_KNOBS})
            if si not in best_y or y_ms < best_y[si][0]:
                best_y[si] = (y_ms, {k: cfg[k] for k in Y_KNOBS})
    sim.sync_status()
    sim.close()
    if not best_x:
        raise RuntimeError("no tuning candidate is valid for %dx%d" % (nx, ny))
    si = min(best_x, key=lambda s: best_x[s][0] + best_y[s][0])
    tuning = dict(shared[si])
    tuning.update(best_x[si][1])
    tuning.update(best_y[si][1])
    out = {"tuning": tuning, "x_ms": best_x[si][0], "y_ms": best_y[si][0]}
    if use_cache:
        cache = _load_cache()
        cache[key] = out
        _store_cache(cache)
    return out


def apply(sim, fp64: str = "auto", **kw) -> Dict:
    """Tune for sim's grid shape (cached) and set the result on the handle."""
    res = tune(sim.nx, sim.ny, fp64=fp64, **kw)
    sim.set_tuning(**res["tuning"])
    return res
