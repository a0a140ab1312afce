"""Run one synthetic forward case through the C ABI and report per-kernel times.

  python -m paper_2006_10142_gb300.run_case --nx 16384 --ny 2048 --steps 4
  python -m paper_2006_10142_gb300.run_case --nx 16384 --ny 16384 --medium const \
      --configs '[{"cols_per_cta": 16}, {"cta_threads": 512}]'

The problem is the seeded heterogeneous medium with a Ricker point source
(the recipe of ``inputs.ricker_problem``) on an nx x ny grid of the unit
square, or, with ``--medium const``, c = 1 (timing only: the kernels do the
same work for any m).  ``--configs`` runs a list of tunings on the same
inputs; every entry prints one JSON line.  Useful for profiling one kernel
shape on a small device footprint and for tuning sweeps.

  python -m paper_2006_10142_gb300.run_case --nx 1024 --ny 1024 --adjoint --steps 100

``--adjoint`` records a run of ``--steps`` steps with 64 receivers along
y = 0.1 and checkpoints every ``--every`` steps, then computes the gradient
of the misfit against zero data once and reports its time per step.
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np

TUNING_KEYS = ("chunk_x", "chunk_y", "rows_per_cta", "cols_per_cta", "pcr_size", "use_graph",
               "solver", "cta_threads", "cta_threads_y", "y_stage", "persist", "x_stage",
               "x_cluster")


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, required=True)
    ap.add_argument("--ny", type=int, required=True)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--medium", choices=["seeded", "const"], default="seeded")
    ap.add_argument("--cfl", type=float, default=0.5,
                    help="tau = cfl h / max c; above 3 the elimination switches to FP64")
    ap.add_argument("--fp64", choices=["auto", "never", "always"], default="auto",
                    help="FP64 elimination: when dominance is weak (auto), never, always")
    ap.add_argument("--adjoint", action="store_true",
                    help="time one gradient (adjoint sweep) after a recorded run")
    ap.add_argument("--every", type=int, default=50, help="checkpoint interval of --adjoint")
    ap.add_argument("--configs", type=str, default=None,
                    help="JSON list of tuning dicts to run one after the other")
    for k in TUNING_KEYS:
        ap.add_argument("--" + k, type=int, default=0)
    args = ap.parse_args(argv)

    import torch
    from . import api, inputs

    dev = torch.device("cuda:0")
    nx, ny = args.nx, args.ny
    if args.medium == "const":
        m_d = torch.ones((ny, nx), dtype=torch.float32, device=dev)
        mmax = 1.0
    else:
        m = inputs.m_field(nx, ny, args.seed, dtype=np.float32)
        m_d = torch.from_numpy(m).to(dev)
        mmax = float(m.max())
    h = min(1.0 / (nx + 1), 1.0 / (ny + 1))
    tau = args.cfl * h / math.sqrt(mmax)
    configs = json.loads(args.configs) if args.configs else [
        {k: getattr(args, k) for k in TUNING_KEYS}]
    total = (args.warmup + args.steps) * len(configs)
    wav = torch.from_numpy(inputs.wavelet_samples(total + 2, tau).astype(np.float32)).to(dev)
    src = (inputs.nearest_node(0.5, nx), inputs.nearest_node(0.5, ny))
    sim = api.AdiWave(m_d, torch.zeros_like(m_d), tau, src=src, wavelet=wav, fp64=args.fp64)
    pts = nx * ny
    for cfg in configs:
        try:
            sim.set_tuning(**cfg)
        except api.AdiError as e:
            print(json.dumps({"nx": nx, "ny": ny, "config": cfg, "error": str(e)}))
            continue
        if args.adjoint:
            print(json.dumps(_adjoint_case(sim, args, src, wav, dev)), flush=True)
            continue
        sim.run(args.warmup, src=src, wavelet=wav)
        sim.sync_status()
        sim.profile(True)
        sim.profile_read()
        sim.run(args.steps, src=src, wavelet=wav)
        ms, cnt = sim.profile_read()
        sim.profile(False)
        sim.sync_status()
        out = {"nx": nx, "ny": ny, "steps": args.steps, "cfl": args.cfl, "fp64": args.fp64,
               "config": cfg,
               "tuning": sim.tuning(),
               "x_ms": ms[0] / max(cnt[0], 1), "y_ms": ms[1] / max(cnt[1], 1)}
        out["x_gbs"] = 12 * pts / (out["x_ms"] * 1e-3) / 1e9
        out["y_gbs"] = 20 * pts / (out["y_ms"] * 1e-3) / 1e9
        out["step_gbs_32B"] = 32 * pts / ((out["x_ms"] + out["y_ms"]) * 1e-3) / 1e9
        print(json.dumps(out), flush=True)
    sim.close()


def _adjoint_case(sim, args, src, wav, dev):
    import torch
    from . import inputs
    nx, ny = args.nx, args.ny
    iy = inputs.nearest_node(0.1, ny)
    rec = np.array([[min(nx - 1, int((r + 0.5) * nx / 64)), iy] for r in range(64)], dtype=np.int32)
    sim.reset(torch.zeros((ny, nx), dtype=torch.float32, device=dev))
    sim.set_checkpointing(args.every)
    tr = sim.run(args.steps, src=src, wavelet=wav, rec=rec)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    gm, _ = sim.adjoint(tr, ckpt_every=args.every)
    e1.record()
    torch.cuda.synchronize()
    sim.sync_status()
    return {"nx": nx, "ny": ny, "steps": args.steps, "every": args.every, "tuning": sim.tuning(),
            "adjoint_ms_per_step": e0.elapsed_time(e1) / args.steps,
            "grad_m_finite": bool(torch.isfinite(gm).all().item())}


if __name__ == "__main__":
    main()
