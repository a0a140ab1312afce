"""Autotuner for the line-solver launch parameters of one grid shape.

Knobs (see ``adi_wave_tuning`` in include/adiwave.h): systems (rows) per CTA
of the x sweep, unknowns per thread in each sweep, strip width of the y sweep,
threads per CTA, the interface solver (warp-shuffle block CR + PCR, or
shared-memory CR handing `pcr_size` equations to warp PCR -- the CR-to-PCR
switch level) and graph replay.

Each candidate runs a few steps of a c = 1 problem of the requested shape
(the kernels do the same work for any coefficient) with per-kernel CUDA
events on the launching stream.  The x-sweep and y-sweep knobs act on
different kernels: for each setting of the shared knobs (solver, CR-to-PCR
switch) the x candidates are timed with the y sweep on automatic, then the
y candidates with the best x.  The planner's automatic choice is timed
first and kept unless a searched tuning is faster (an empty tuning dict
means "automatic").  Results are cached per (device, nx, ny, precision) in a JSON file
(``$ADIWAVE_TUNE_CACHE`` or ``~/.cache/adiwave/tuning.json``).
"""
from __future__ import annotations

import itertools
import json
import os
from typing import Dict

X_KNOBS = ("chunk_x", "rows_per_cta", "cta_threads", "x_stage", "x_cluster")
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
    # stage 3 = the TMA-pipelined persistent sweeps, 2 = direct loads (x) or
    # L2 prefetch (y), 1 = shared-memory staging, 4 = (y only) persistent CTAs
    # whose column segments meet through global memory, 5 = (x only) the band
    # form, each row over a cluster of x_cluster CTAs
    xs = [dict(chunk_x=k, rows_per_cta=0, cta_threads=t, x_stage=s, x_cluster=0)
          for k, t, s in itertools.product((8, 16, 32), (256, 512, 1024), (3, 2))]
    xs += [dict(chunk_x=k, rows_per_cta=0, cta_threads=0, x_stage=5, x_cluster=c)
           for k, c in itertools.product((32, 16), (2, 4))]
    ys = [dict(chunk_y=k, cols_per_cta=w, cta_threads_y=t, y_stage=s)
          for k, w, t, s in itertools.product((8, 16, 32), (8, 16), (256, 512, 1024), (4, 3, 1, 2))]
    return shared, xs, ys


def search(measure, shared, xs, ys):
    """(total ms, tuning, x_ms, y_ms) of the best setting, or None.

    measure(cfg) returns (x_ms, y_ms) or None when the shape rejects cfg.
    The planner's own choice (the empty tuning, all knobs automatic) is the
    reference: a searched tuning replaces it only when it is faster.  For
    each shared setting the x knobs are chosen by the x time with the y
    sweep on automatic, then the y knobs by the y time with that x."""
    ref = measure({})
    best = (ref[0] + ref[1], {}, ref[0], ref[1]) if ref else None
    for sh in shared:
        bx = None
        for xc in xs:
            cfg = dict(sh)
            cfg.update(xc)
            r = measure(cfg)
            if r and (bx is None or r[0] < bx[0]):
                bx = (r[0], xc)
        if bx is None:
            continue
        by = None
        for yc in ys:
            cfg = dict(sh)
            cfg.update(bx[1])
            cfg.update(yc)
            r = measure(cfg)
            if r and (by is None or r[1] < by[0]):
                by = (r[1], yc)
        if by is None:
            continue
        tot = bx[0] + by[0]
        if best is None or tot < best[0]:
            t = dict(sh)
            t.update(bx[1])
            t.update(by[1])
            best = (tot, t, bx[0], by[0])
    return best


def tune(nx: int, ny: int, fp64: str = "auto", steps: int = 3, warmup: int = 1,
         use_cache: bool = True, verbose: bool = False) -> Dict:
    """Best tuning for an nx x ny grid: {'tuning': {...}, 'x_ms': .., 'y_ms': ..}."""
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

    def measure(cfg):
        """(x_ms, y_ms) of one tuning, or None when the shape rejects it."""
        try:
            sim.set_tuning(**cfg)
        except api.AdiError:
            return None
        sim.run(warmup)
        sim.profile(True)
        sim.profile_read()
        sim.run(steps)
        ms, cnt = sim.profile_read()
        sim.profile(False)
        r = (ms[0] / max(cnt[0], 1), ms[1] / max(cnt[1], 1))
        if verbose:
            print(json.dumps({"cfg": cfg, "x_ms": r[0], "y_ms": r[1]}))
        return r

    best = search(measure, shared, xs, ys)
    sim.sync_status()
    sim.close()
    if best is None:
        raise RuntimeError("no tuning candidate is valid for %dx%d" % (nx, ny))
    out = {"tuning": best[1], "x_ms": best[2], "y_ms": best[3]}
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
