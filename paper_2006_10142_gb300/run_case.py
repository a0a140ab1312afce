"""Run one synthetic forward case through the C ABI and report per-kernel times.

  python -m paper_2006_10142_gb300.run_case --nx 16384 --ny 2048 --steps 4

The problem is the seeded heterogeneous medium with a Ricker point source
(the recipe of ``inputs.ricker_problem``) on an nx x ny grid of the unit
square.  Useful for profiling one kernel shape on a small device footprint.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, required=True)
    ap.add_argument("--ny", type=int, required=True)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--seed", type=int, default=0)
    for k in ("chunk_x", "chunk_y", "rows_per_cta", "cols_per_cta", "pcr_size", "use_graph",
              "solver"):
        ap.add_argument("--" + k, type=int, default=0)
    args = ap.parse_args(argv)

    import torch
    from . import api, inputs

    dev = torch.device("cuda:0")
    nx, ny = args.nx, args.ny
    m = inputs.m_field(nx, ny, args.seed, dtype=np.float32)
    h = min(1.0 / (nx + 1), 1.0 / (ny + 1))
    tau = 0.5 * h / math.sqrt(float(m.max()))
    total = args.warmup + args.steps
    wav = torch.from_numpy(inputs.wavelet_samples(total + 2, tau).astype(np.float32)).to(dev)
    src = (inputs.nearest_node(0.5, nx), inputs.nearest_node(0.5, ny))
    m_d = torch.from_numpy(m).to(dev)
    sim = api.AdiWave(m_d, torch.zeros_like(m_d), tau, src=src, wavelet=wav)
    tun = {k: getattr(args, k) for k in ("chunk_x", "chunk_y", "rows_per_cta", "cols_per_cta",
                                          "pcr_size", "use_graph", "solver")}
    if any(tun.values()):
        sim.set_tuning(**tun)
    sim.run(args.warmup, src=src, wavelet=wav)
    sim.sync_status()
    sim.profile(True)
    sim.profile_read()
    sim.run(args.steps, src=src, wavelet=wav)
    ms, cnt = sim.profile_read()
    sim.sync_status()
    pts = nx * ny
    out = {"nx": nx, "ny": ny, "steps": args.steps, "tuning": sim.tuning(),
           "x_ms": ms[0] / max(cnt[0], 1), "y_ms": ms[1] / max(cnt[1], 1)}
    out["x_gbs"] = 12 * pts / (out["x_ms"] * 1e-3) / 1e9
    out["y_gbs"] = 20 * pts / (out["y_ms"] * 1e-3) / 1e9
    print(json.dumps(out))
    sim.close()


if __name__ == "__main__":
    main()
