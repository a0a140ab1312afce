#!/usr/bin/env python3
"""Benchmark of the implicit ADI wave-equation hot path on GB300.

One bench step = one pass of the hot path over one synthetic problem: the
start-up (Eq. CN2) followed by the workload's ADI time steps (RHS assembly,
x sweep, y sweep + update, Algorithm 1's loop), with every input resident in
HBM.  The default workload is the 16384 x 16384 bandwidth case: seeded
heterogeneous c-field, Ricker point source, tau = 0.5 h / max c, 200 time
steps, four FP32 fields of 1 GiB each resident (far larger than L2, so no
flush is needed between steps).

Prints ONE JSON line (rank 0).  `value` is whole-job grid-point updates per
second over the timed region (the library's own time loop, step pairs
replayed from CUDA graphs; CUDA events on the launching stream, max over
ranks).  A second timed region of the same steps records a CUDA event pair
around every launch (direct launches): `roofline` reports the dominant
kernel's algorithmic HBM bytes per launch over its average duration there,
against the measured copy bandwidth.  `e2e` is the same metric from pinned
host buffers (H2D of m, phi and the wavelet, D2H of the final field inside
the timed region).  `cpu_baseline` is the FP64 oracle timed on the host cores
on a bounded sample of the same workload.  The default line also carries an
`adjoint` sub-record (adjoint_1024: gradient time per time step) and a
`batch` sub-record (batch_64_shots: one persistent launch per step against
the plain kernels launched per shot).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload ricker_16384|ricker_4096|standing_wave_128|
                              batch_64_shots|adjoint_1024|custom]
  python bench.py --workload custom --nx 4096 --ny 16384 --time-steps 2 \
                  [--medium seeded|const] [--cfl 0.5] [--fp64 auto|never|always]
                  [--tuning '{"chunk_y": 32}']
With --gpus N > 1 and no torchrun environment, bench.py starts N ranks itself
(torch.distributed.run on 127.0.0.1).  Every rank runs its own replica of a
single-grid workload on its own GPU (a single grid does not shard); the
batched workload shards its shots over the ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import socket
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "ricker_16384": dict(n=16384, time_steps=200, kind="ricker"),
    "ricker_4096": dict(n=4096, time_steps=1000, kind="ricker"),
    "standing_wave_128": dict(n=128, time_steps=200, kind="standing"),
    "batch_64_shots": dict(count=64, time_steps=500, kind="batch"),
    "adjoint_1024": dict(n=1024, time_steps=2000, n_rec=64, ckpt_every=50, kind="adjoint"),
    "custom": dict(kind="custom"),
}
DEFAULT_WORKLOAD = "ricker_16384"
METRIC = "ADI grid-point updates/sec"
UNIT = "grid-point updates/s"
# algorithmic HBM bytes per grid point per launch (FP32 fields)
BYTES_X = 12  # read u^k, m; write w
BYTES_Y = 20  # read w, m, u^k, u^{k-1}; write u^{k+1}
# dram__bytes_read.sum + dram__bytes_write.sum per 16384^2 launch, measured by
# ncu on a smaller grid with the same launch shape and scaled by the number of
# grid points (profiles/).  Only valid for the 16384^2 workload and the
# kernel builds the captures were taken on; None once a kernel has changed.
NCU_TRAFFIC = {("ricker_16384", "y_coop_kernel"): 5702261248,
               ("ricker_16384", "x_band_kernel"): 3124610560}


def measured_peak_gbs():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        return self.parse(self.lines)

    @staticmethod
    def parse(lines):
        """Median SM clock, max clock and the throttle reasons seen in
        `nvidia-smi --format=csv,noheader,nounits` lines of FIELDS."""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() in ("active", "1", "0x1"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# command line and rank start-up
# ---------------------------------------------------------------------------
def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-sub", action="store_true",
                    help="leave out the adjoint and batch sub-records of the default line")
    # --workload custom: one forward grid of any shape (profiling, tuning)
    ap.add_argument("--nx", type=int, default=0)
    ap.add_argument("--ny", type=int, default=0)
    ap.add_argument("--time-steps", type=int, default=0,
                    help="ADI time steps per bench step (default: the workload's)")
    ap.add_argument("--medium", choices=["seeded", "const"], default="seeded")
    ap.add_argument("--cfl", type=float, default=0.5,
                    help="tau = cfl h / max c; above about 3 the elimination switches to FP64")
    ap.add_argument("--fp64", choices=["auto", "never", "always"], default="auto")
    ap.add_argument("--tuning", type=str, default=None,
                    help="JSON dict of adi_wave_tuning fields (replaces the autotuner)")
    ap.add_argument("--print-ranks", action="store_true",
                    help="print this process's RANK / WORLD_SIZE and exit (launcher check)")
    args = ap.parse_args(argv)
    if args.workload == "custom" and (args.nx < 1 or args.ny < 1):
        ap.error("--workload custom needs --nx and --ny")
    return args


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def spawn_ranks(args, argv):
    """With --gpus N > 1 outside torchrun: run N ranks of this script under
    torch.distributed.run on 127.0.0.1 and return its exit code, else None."""
    if args.gpus <= 1 or "WORLD_SIZE" in os.environ:
        return None
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           "--nproc-per-node=%d" % args.gpus, "--master-addr=127.0.0.1",
           "--master-port=%d" % _free_port(), os.path.abspath(__file__)] + list(argv)
    return subprocess.run(cmd).returncode


# ---------------------------------------------------------------------------
# problems
# ---------------------------------------------------------------------------
class Problem:
    """One single-grid forward problem, FP32 inputs on the host."""

    def __init__(self, nx, ny, m, phi, tau, src, wavelet, time_steps, medium, source):
        self.nx, self.ny, self.m, self.phi, self.tau = nx, ny, m, phi, tau
        self.src, self.wavelet, self.time_steps = src, wavelet, time_steps
        self.medium, self.source = medium, source


def make_problem(wl, args):
    from paper_2006_10142_gb300 import inputs
    ts = args.time_steps or wl.get("time_steps", 2)
    if wl["kind"] == "standing":
        n = wl["n"]
        p = inputs.standing_wave_problem(n, ts)
        return Problem(n, n, p.m.astype(np.float32), p.phi.astype(np.float32), p.tau, None, None,
                       ts, "c = 1", "none")
    if wl["kind"] == "ricker":
        n = wl["n"]
        p = inputs.ricker_problem(n, ts, seed=0, m_dtype=np.float32)
        return Problem(n, n, p.m, p.phi.astype(np.float32), p.tau, p.src,
                       p.wavelet.astype(np.float32), ts,
                       "seeded c-field 1 + 2 sigmoid(8 Gaussian bumps), m = c^2", "Ricker f=20")
    # custom: the same recipe (or c = 1) on an nx x ny grid of the unit square
    nx, ny = args.nx, args.ny
    if args.medium == "const":
        m = np.ones((ny, nx), dtype=np.float32)
        medium = "c = 1"
    else:
        m = inputs.m_field(nx, ny, 0, dtype=np.float32)
        medium = "seeded c-field 1 + 2 sigmoid(8 Gaussian bumps), m = c^2"
    h = min(1.0 / (nx + 1), 1.0 / (ny + 1))
    tau = args.cfl * h / float(np.sqrt(m.max()))
    src = (inputs.nearest_node(0.5, nx), inputs.nearest_node(0.5, ny))
    wav = inputs.wavelet_samples(ts + 2, tau).astype(np.float32)
    return Problem(nx, ny, m, np.zeros((ny, nx), dtype=np.float32), tau, src, wav, ts, medium,
                   "Ricker f=20")


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------
def _oracle_start(prob):
    import oracle
    m64 = prob.m.astype(np.float64)
    hx, hy = 1.0 / (prob.nx + 1), 1.0 / (prob.ny + 1)
    u0, u1 = oracle.adi_init(m64, prob.phi.astype(np.float64), hx, hy, prob.tau)
    wav = prob.wavelet.astype(np.float64) if prob.wavelet is not None else None
    return m64, hx, hy, u0, u1, wav


def cpu_baseline(prob, budget_s=15.0):
    """FP64 oracle on the host cores, on a bounded sample: the workload's grid,
    a few of its time steps from the same start (steps scaled to the budget)."""
    import oracle
    threads = os.cpu_count() or 1
    m64, hx, hy, u0, u1, wav = _oracle_start(prob)
    t0 = time.perf_counter()
    up, uc, _ = oracle.adi_run(m64, u0, u1, hx, hy, prob.tau, 1, k0=1, src=prob.src, wavelet=wav,
                               threads=threads)
    t1 = time.perf_counter() - t0
    extra = int(max(0, min(prob.time_steps - 1, budget_s / max(t1, 1e-6) - 1)))
    steps = 1
    t_total = t1
    if extra > 0:
        t0 = time.perf_counter()
        oracle.adi_run(m64, up, uc, hx, hy, prob.tau, extra, k0=2, src=prob.src, wavelet=wav,
                       threads=threads)
        t_total += time.perf_counter() - t0
        steps += extra
    pts = prob.nx * prob.ny
    return {"value": float(pts * steps / t_total), "unit": UNIT, "cores": threads,
            "kind": "oracle",
            "sample": "%d of the workload's %d ADI steps on the full %dx%d grid, FP64, %d threads"
                      % (steps, prob.time_steps, prob.nx, prob.ny, threads)}


def run_reference(args, wl, rank):
    """The reference arm: the FP64 oracle as it stands, on the host cores,
    each bench step a bounded sample of the workload."""
    if rank != 0:
        return None
    import oracle
    from paper_2006_10142_gb300 import inputs
    threads = os.cpu_count() or 1
    if wl["kind"] == "batch":
        # a sample of the batch: a few steps of every shot of one size class
        sizes = inputs.batch_sizes(wl["count"], seed=0)
        shots = [b for b in range(len(sizes)) if sizes[b] == min(sizes)][:4]
        probs = [inputs.ricker_problem(sizes[b], wl["time_steps"], seed=b, m_dtype=np.float32)
                 for b in shots]
        sample_steps = 2
        states = []
        for p in probs:
            q = Problem(p.n, p.n, p.m, p.phi.astype(np.float32), p.tau, p.src,
                        p.wavelet.astype(np.float32), wl["time_steps"], "", "")
            m64, hx, hy, u0, u1, wav = _oracle_start(q)
            states.append([q, m64, hx, hy, wav, u0, u1, 1])

        def one():
            for st in states:
                q, m64, hx, hy, wav, up, uc, k = st
                up, uc, _ = oracle.adi_run(m64, up, uc, hx, hy, q.tau, sample_steps, k0=k,
                                           src=q.src, wavelet=wav, threads=threads)
                st[5], st[6], st[7] = up, uc, k + sample_steps

        pts = sum(st[0].nx * st[0].ny for st in states) * sample_steps
        sample = ("%d ADI steps of %d of the %d shots (n = %d) per bench step, FP64, %d threads"
                  % (sample_steps, len(states), len(sizes), min(sizes), threads))
        metric, unit, hib, dtype = METRIC, UNIT, True, "f64"
        conv = lambda dt: pts * args.steps / dt
        cfg = {"workload": args.workload, "shots": len(sizes), "time_steps": wl["time_steps"]}
    elif wl["kind"] == "adjoint":
        n = wl["n"]
        prob, _ = inputs.adjoint_problem(n, wl["time_steps"], seed=0, n_rec=wl["n_rec"])
        sample_steps = 4
        m64 = prob.m.astype(np.float32).astype(np.float64)
        hx = 1.0 / (n + 1)
        z = np.zeros((n, n))
        wav = prob.wavelet.astype(np.float32).astype(np.float64)
        resid = np.full((sample_steps, prob.rec.shape[0]), 1e-3)

        def one():
            oracle.adi_adjoint(m64, z, z, hx, hx, prob.tau, sample_steps, resid, prob.rec, k0=1,
                               src=prob.src, wavelet=wav, threads=threads)

        sample = ("gradient of a %d-step run of the %dx%d grid per bench step (of the workload's "
                  "%d), FP64, %d threads" % (sample_steps, n, n, wl["time_steps"], threads))
        metric, unit, hib, dtype = "adjoint gradient time/step", "ms", False, "f64"
        conv = lambda dt: 1e3 * dt / args.steps / sample_steps
        cfg = {"workload": args.workload, "n": n, "time_steps": wl["time_steps"]}
    else:
        prob = make_problem(wl, args)
        m64, hx, hy, u0, u1, wav = _oracle_start(prob)
        pts = prob.nx * prob.ny
        sample_steps = max(1, min(prob.time_steps, int(2e8 // pts) or 1))
        state = [u0, u1, 1]

        def one():
            up, uc, k = state
            up, uc, _ = oracle.adi_run(m64, up, uc, hx, hy, prob.tau, sample_steps, k0=k,
                                       src=prob.src, wavelet=wav, threads=threads)
            state[0], state[1], state[2] = up, uc, k + sample_steps

        sample = ("%d ADI steps of the %dx%d grid per bench step (of the workload's %d), FP64, "
                  "%d threads" % (sample_steps, prob.nx, prob.ny, prob.time_steps, threads))
        metric, unit, hib, dtype = METRIC, UNIT, True, "f64"
        conv = lambda dt: pts * sample_steps * args.steps / dt
        cfg = {"workload": args.workload, "nx": prob.nx, "ny": prob.ny,
               "time_steps": prob.time_steps}

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    val = conv(dt)
    return {"metric": metric, "value": val, "unit": unit, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": hib,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
            "impl": "reference", "config": cfg,
            "cpu_baseline": {"value": val, "unit": unit, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# ---------------------------------------------------------------------------
# timing helpers
# ---------------------------------------------------------------------------
def _clock_sampler(ctx):
    vis = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    lr = ctx["local_rank"]
    return ClockSampler(vis[lr].strip() if lr < len(vis) else lr)


def _timed(ctx, step_fn, launch_count, steps=None, sample_clocks=True):
    """K steps between barriers + syncs, timed by CUDA events on the launching
    stream; returns (max_ms over ranks, own ms, launches, clocks)."""
    import torch
    args, world, rank, dist = ctx["args"], ctx["world"], ctx["rank"], ctx["dist"]
    steps = args.steps if steps is None else steps
    stream = torch.cuda.current_stream()
    clocks = _clock_sampler(ctx)
    if rank == 0 and sample_clocks:
        clocks.start()
        time.sleep(0.5)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        step_fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = launch_count() - l0
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if (rank == 0 and sample_clocks) else None
    ms = ev0.elapsed_time(ev1)
    return _max_over_ranks(ctx, ms), ms, launches, clk


def _max_over_ranks(ctx, v):
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=ctx["dev"])
    if ctx["world"] > 1:
        ctx["dist"].all_reduce(t, op=ctx["dist"].ReduceOp.MAX)
    return float(t.item())


def _roofline(kms, kcnt, kinds, alg_bytes, workload=None):
    """Dominant kernel's algorithmic GB/s against the measured copy bandwidth."""
    peak, peak_kind = measured_peak_gbs()
    k = max(kinds, key=lambda q: kms[q])
    per_launch_ms = kms[k] / max(kcnt[k], 1)
    achieved = alg_bytes[k] / (per_launch_ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": kinds[k], "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
            "traffic": NCU_TRAFFIC.get((workload, kinds[k])), "alg_bytes_per_launch": alg_bytes[k],
            "avg_launch_ms": per_launch_ms,
            "kernel_ms": {kinds[q]: kms[q] for q in kinds},
            "kernel_launches": {kinds[q]: kcnt[q] for q in kinds}}


def _profiled(ctx, step_fn, handle):
    """The same K steps with a CUDA event pair around every launch (direct
    launches, no graphs): per-kind total ms and launch counts."""
    handle.sync_status()
    handle.profile(True)
    handle.profile_read()
    max_ms, _, _, _ = _timed(ctx, step_fn, handle.launch_count, sample_clocks=False)
    kms, kcnt = handle.profile_read()
    handle.profile(False)
    handle.sync_status()
    return max_ms, kms, kcnt


# ---------------------------------------------------------------------------
# GPU arms
# ---------------------------------------------------------------------------
def run_single(ctx, prob):
    """One grid, the library's time loop (adi_wave_run) per bench step."""
    import torch
    from paper_2006_10142_gb300 import api, autotune
    args, world, rank, dev = ctx["args"], ctx["world"], ctx["rank"], ctx["dev"]
    nx, ny, ts = prob.nx, prob.ny, prob.time_steps
    pts = nx * ny
    m_d = torch.from_numpy(prob.m).to(dev)
    phi_d = torch.from_numpy(prob.phi).to(dev)
    src = prob.src
    wav_d = torch.from_numpy(prob.wavelet).to(dev) if prob.wavelet is not None else None
    h = api.AdiWave(m_d, phi_d, prob.tau, src=src, wavelet=wav_d, fp64=args.fp64)
    tuned = None
    if args.tuning:
        h.set_tuning(**json.loads(args.tuning))
    elif not args.no_autotune:
        tuned = autotune.apply(h, fp64=args.fp64, steps=2, warmup=1)

    def bench_step():
        h.reset(phi_d)
        h.run(ts, src=src, wavelet=wav_d)

    for _ in range(max(args.warmup, 0)):
        bench_step()
    h.sync_status()
    max_ms, _, launches, clk = _timed(ctx, bench_step, h.launch_count)
    h.sync_status()
    value = world * pts * ts * args.steps / (max_ms / 1e3)
    # the same steps again with an event pair around every kernel launch
    prof_ms, kms, kcnt = _profiled(ctx, bench_step, h)
    tun = h.tuning()
    # the kernels the plan launches: the TMA-pipelined forms (stage 3) or the
    # one-CTA-per-tile forms
    xname = {3: "x_pipe_kernel", 5: "x_band_kernel"}.get(tun.get("x_stage"), "x_sweep_kernel")
    yname = {3: "y_pipe_kernel", 4: "y_coop_kernel"}.get(tun.get("y_stage"), "y_sweep_kernel")
    roof = _roofline(kms, kcnt, {0: xname, 1: yname}, {0: BYTES_X * pts, 1: BYTES_Y * pts},
                     args.workload)
    roof["step_gbs_32B"] = 32.0 * pts * ts * args.steps / (max_ms / 1e3) / 1e9
    roof["timed_region"] = ("second timed region of the same K bench steps, a CUDA event pair "
                            "around every launch (direct launches, no graphs): %.3f ms per bench "
                            "step against %.3f ms with graphs" % (prof_ms / args.steps,
                                                                   max_ms / args.steps))

    e2e = None
    if not args.no_e2e:
        e2e = _e2e(ctx, h, prob, m_d, phi_d, wav_d)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob)
    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "nx": nx, "ny": ny, "time_steps": ts,
                       "medium": prob.medium, "source": prob.source,
                       "l2": ("inputs larger than L2 (4 FP32 fields of %.0f MiB)" % (pts * 4 / 2**20)
                              if pts * 16 > 2 * 129e6 else "inputs smaller than L2: no flush, "
                              "steps of one run reuse L2-resident fields"),
                       "timed_launches": "adi_wave_run: step pairs replayed from CUDA graphs",
                       "e2e_copies": "per bench step: H2D of m, phi, wavelet from pinned host memory "
                                     "(torch copy_ on a copy stream into a second device set) and "
                                     "D2H of u^{S+1}, overlapping the neighbouring steps' compute; "
                                     "the library calls take the device copies",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "tuning": tun, "autotuned": tuned is not None,
                       "fp64": args.fp64},
            "roofline": roof, "gpu_launches": int(launches), "clocks": clk, "e2e": e2e,
            "cpu_baseline": cpu,
        }
    h.close()
    return out


def _e2e(ctx, h, prob, m_d, phi_d, wav_d):
    """The metric end to end: every bench step uploads its inputs from pinned
    host memory, runs, and reads its result back.  The copies run on their
    own streams: the upload of step i + 1 (into the other of two device input
    sets) and the read-back of step i overlap the compute of the neighbouring
    steps."""
    import torch
    args, world = ctx["args"], ctx["world"]
    nx, ny, ts, src = prob.nx, prob.ny, prob.time_steps, prob.src
    m_h = torch.from_numpy(prob.m).pin_memory()
    phi_h = torch.from_numpy(prob.phi).pin_memory()
    wav_h = torch.from_numpy(prob.wavelet).pin_memory() if prob.wavelet is not None else None
    out_h = torch.empty((ny, nx), dtype=torch.float32).pin_memory()
    comp = torch.cuda.current_stream()
    up_st, down_st = torch.cuda.Stream(), torch.cuda.Stream()
    sets = [(torch.empty_like(m_d), torch.empty_like(phi_d),
             torch.empty_like(wav_d) if wav_d is not None else None) for _ in range(2)]
    uploaded = [torch.cuda.Event() for _ in range(2)]
    consumed = [torch.cuda.Event() for _ in range(2)]
    done = torch.cuda.Event()

    def upload(i):
        m_s, phi_s, wav_s = sets[i % 2]
        with torch.cuda.stream(up_st):
            up_st.wait_event(consumed[i % 2])
            m_s.copy_(m_h, non_blocking=True)
            phi_s.copy_(phi_h, non_blocking=True)
            if wav_s is not None:
                wav_s.copy_(wav_h, non_blocking=True)
            uploaded[i % 2].record(up_st)

    def e2e_steps(k):
        for q in range(2):
            consumed[q].record(comp)
        upload(0)
        for i in range(k):
            m_s, phi_s, wav_s = sets[i % 2]
            comp.wait_event(uploaded[i % 2])
            h.reset(phi_s, m=m_s, stream=comp)
            h.run(ts, src=src, wavelet=wav_s, stream=comp)
            consumed[i % 2].record(comp)  # the run reads the wavelet until it ends
            if i + 1 < k:
                upload(i + 1)
            _, uc, _ = h.state(stream=comp)
            done.record(comp)
            with torch.cuda.stream(down_st):
                down_st.wait_event(done)
                out_h.copy_(uc, non_blocking=True)
            uc.record_stream(down_st)
        torch.cuda.synchronize()

    e2e_steps(2)
    if world > 1:
        ctx["dist"].barrier()
    t0 = time.perf_counter()
    e2e_steps(args.steps)
    e_dt = _max_over_ranks(ctx, time.perf_counter() - t0)
    if not torch.equal(out_h, h.state()[1].cpu()):
        raise RuntimeError("e2e read-back differs from the final device state")
    bi = m_h.numel() * 4 + phi_h.numel() * 4 + (wav_h.numel() * 4 if wav_h is not None else 0)
    return {"value": world * nx * ny * ts * args.steps / e_dt, "unit": UNIT,
            "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(nx * ny * 4)}


def run_batch(ctx, steps=None):
    """64 shots with n from {256, 512, 1024, 2048} in the default batch mode
    (per-shot chains of the single-grid kernels on parallel graph branches);
    the one-launch persistent kernel and the serial per-shot launches are timed
    beside it."""
    import torch
    from paper_2006_10142_gb300 import api, inputs, shard
    args, world, rank, dev = ctx["args"], ctx["world"], ctx["rank"], ctx["dev"]
    wl = WORKLOADS["batch_64_shots"]
    ts = args.time_steps or wl["time_steps"] if args.workload == "batch_64_shots" else wl["time_steps"]
    K = args.steps if steps is None else steps
    sizes_all = inputs.batch_sizes(wl["count"], seed=0)
    mine = shard.local_shots([(s, s) for s in sizes_all], rank, world)
    probs = [inputs.ricker_problem(sizes_all[b], ts, seed=b, m_dtype=np.float32) for b in mine]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    ms_ = [t(p.m) for p in probs]
    phis = [t(p.phi) for p in probs]
    wavs = [t(p.wavelet) for p in probs]
    srcs = [p.src for p in probs]
    B = api.AdiWaveBatch(ms_, phis, [p.tau for p in probs])
    pts = sum(p.n * p.n for p in probs)
    pts_all = sum(s * s for s in sizes_all)

    def bench_step():
        B.reset(phis)
        B.run(ts, srcs=srcs, wavelets=wavs)

    for _ in range(max(args.warmup, 0)):
        bench_step()
    B.sync_status()
    max_ms, _, launches, clk = _timed(ctx, bench_step, B.launch_count, steps=K)
    B.sync_status()
    # the shots' kernels run concurrently, so a per-launch duration says
    # little: the roofline here is the whole batched step's (all shots' x and
    # y sweeps, 32 algorithmic bytes per point) over the wall time
    peak, peak_kind = measured_peak_gbs()
    ach = 32.0 * pts_all * ts * K / (max_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "kernel": "batched step (every shot's x and y sweeps)",
            "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
            "peak_source": peak_kind, "traffic": None,
            "alg_bytes_per_step": 32 * pts_all, "timed_region": "wall time of the timed region"}
    # the same work in the other batch modes: the one-launch persistent
    # kernel (mode 0) and the plain kernels launched serially per shot (mode 1)
    other = {}
    for mode in (0, 1):
        B.set_mode(mode)
        for _ in range(2):
            bench_step()
        ms_m, _, _, _ = _timed(ctx, bench_step, B.launch_count, steps=K, sample_clocks=False)
        other[mode] = pts_all * ts * K / (ms_m / 1e3)
    B.set_mode(2)
    B.sync_status()
    B.close()
    value = pts_all * ts * K / (max_ms / 1e3)
    plain = other[1]
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": args.warmup, "ms_per_step": max_ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch_64_shots", "shots": len(sizes_all),
                       "points_per_step": pts_all, "time_steps": ts,
                       "l2": "inputs larger than L2 (%.0f MiB per field over all shots)"
                             % (pts_all * 4 / 2**20),
                       "timed_launches": "batch mode 2: each shot's steps a chain of the "
                                         "single-grid kernels on one of eight streams, step "
                                         "pairs replayed from one CUDA graph per pair",
                       "persistent_kernel_value": other[0],
                       "persistent_over_plain": other[0] / plain,
                       "parallelism": "shot-sharded" if world > 1 else "single GPU",
                       "plain_per_shot_value": plain, "batched_over_plain": value / plain},
            "roofline": roof, "gpu_launches": int(launches), "clocks": clk, "e2e": None,
            "cpu_baseline": None}


def run_adjoint(ctx, steps=None):
    """1024^2, 64 receivers, 2000 steps, checkpoint every 50: time of the
    gradient (adjoint sweep with recomputation) per time step."""
    import torch
    from paper_2006_10142_gb300 import api, inputs
    args, world, dev = ctx["args"], ctx["world"], ctx["dev"]
    wl = WORKLOADS["adjoint_1024"]
    n, every = wl["n"], wl["ckpt_every"]
    ts = args.time_steps or wl["time_steps"] if args.workload == "adjoint_1024" else wl["time_steps"]
    K = args.steps if steps is None else steps
    prob, m_true = inputs.adjoint_problem(n, ts, seed=0, n_rec=wl["n_rec"])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    wav = t(prob.wavelet)
    zeros = torch.zeros((n, n), dtype=torch.float32, device=dev)
    obs = api.AdiWave(t(m_true), zeros, prob.tau, src=prob.src, wavelet=wav)
    d = obs.run(ts, src=prob.src, wavelet=wav, rec=prob.rec)
    obs.close()
    h = api.AdiWave(t(prob.m), zeros, prob.tau, src=prob.src, wavelet=wav)
    h.set_checkpointing(every)
    state = {}

    def forward():
        h.reset(zeros)
        state["tr"] = h.run(ts, src=prob.src, wavelet=wav, rec=prob.rec)

    def grad():
        state["g"] = h.adjoint(state["tr"] - d, ckpt_every=every)

    for _ in range(max(args.warmup, 1)):
        forward()
        grad()
    torch.cuda.synchronize()
    f_ms, _, _, _ = _timed(ctx, forward, h.launch_count, steps=K, sample_clocks=False)
    forward()
    adj_ms, _, launches, clk = _timed(ctx, grad, h.launch_count, steps=K)
    h.sync_status()
    finite = bool(torch.isfinite(state["g"][0]).all().item())
    h.close()
    per_step = adj_ms / K / ts
    return {"metric": "adjoint gradient time/step", "value": per_step, "unit": "ms",
            "n_gpus": world, "steps": K, "warmup": args.warmup,
            "ms_per_step": adj_ms / K, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 gradient sum)",
            "data": "synthetic",
            "config": {"workload": "adjoint_1024", "n": n, "time_steps": ts,
                       "receivers": wl["n_rec"], "ckpt_every": every,
                       "forward_ms_per_time_step": f_ms / K / ts,
                       "adjoint_over_forward": (adj_ms / f_ms) if f_ms > 0 else None,
                       "grad_finite": finite,
                       "l2": "fields of 4 MiB: L2-resident, no flush (the workload's own size)"},
            "roofline": None, "gpu_launches": int(launches), "clocks": clk, "e2e": None,
            "cpu_baseline": None}


def _sub_record(r):
    """The part of a workload's line that a sub-record keeps."""
    keep = ("metric", "value", "unit", "ms_per_step", "steps", "higher_is_better", "config",
            "roofline", "gpu_launches", "clocks")
    return {k: r[k] for k in keep if k in r}


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    args = parse_args(argv)
    rc = spawn_ranks(args, argv)
    if rc is not None:
        sys.exit(rc)
    wl = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.print_ranks:
        print(json.dumps({"rank": rank, "world_size": world, "local_rank": local_rank}), flush=True)
        return

    if args.impl == "reference":
        out = run_reference(args, wl, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    ctx = dict(args=args, wl=wl, world=world, rank=rank, local_rank=local_rank, dev=dev,
               dist=dist)
    if wl["kind"] == "batch":
        out = run_batch(ctx)
    elif wl["kind"] == "adjoint":
        out = run_adjoint(ctx)
    else:
        out = run_single(ctx, make_problem(wl, args))
        if args.workload == DEFAULT_WORKLOAD and not args.no_sub:
            # the rest of the metric on the same GPU: the adjoint's time per
            # step and the batched form against the plain kernels per shot
            sub_ctx = dict(ctx)
            sub_ctx["args"] = argparse.Namespace(**dict(vars(args), time_steps=0))
            adj = run_adjoint(sub_ctx, steps=max(1, min(args.steps, 3)))
            bat = run_batch(sub_ctx, steps=max(1, min(args.steps, 3)))
            if out is not None:
                out["adjoint"] = _sub_record(adj)
                out["batch"] = _sub_record(bat)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
