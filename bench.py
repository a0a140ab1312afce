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
second over the timed region (CUDA events on the launching stream, max over
ranks); `e2e` is the same metric through the public API from pinned host
buffers (H2D of m and phi, D2H of the final field inside the timed region, on
copy streams that overlap the neighbouring steps' compute);
`roofline` reports the dominant kernel's algorithmic HBM bytes per launch over
its average event-timed duration against the measured copy bandwidth;
`cpu_baseline` is the FP64 oracle timed on the host cores on a bounded sample
of the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload ricker_16384|ricker_4096|standing_wave_128]
Under torchrun (N > 1) every rank runs its own replica of the workload on its
own GPU (the single grid does not shard; the batched form shards by shot).
"""
from __future__ import annotations

import argparse
import json
import os
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
}
METRIC = "ADI grid-point updates/sec"
UNIT = "grid-point updates/s"
# algorithmic HBM bytes per grid point per launch (FP32 fields)
BYTES_X = 12  # read u^k, m; write w
BYTES_Y = 20  # read w, m, u^k, u^{k-1}; write u^{k+1}
# dram__bytes_read.sum + dram__bytes_write.sum per 16384^2 launch, measured by
# ncu on a smaller grid with the same launch shape and scaled by the number of
# grid points: y_pipe_kernel on 4096 x 16384 (x 4,
# profiles/y_pipe_kernel_4096x16384.txt), x_pipe_kernel (rows split over CTA
# pairs) on 16384 x 2048 (x 8, profiles/x_pipe_kernel_16384x2048.txt).  Only
# valid for the 16384^2 workload.
NCU_TRAFFIC = {("ricker_16384", "y_pipe_kernel"): 5692224512,
               ("ricker_16384", "x_pipe_kernel"): 2957748224}


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
def make_problem(wl):
    from paper_2006_10142_gb300 import inputs
    n, ts = wl["n"], wl["time_steps"]
    if wl["kind"] == "standing":
        p = inputs.standing_wave_problem(n, ts)
        p.m = p.m.astype(np.float32)
        p.phi = p.phi.astype(np.float32)
        return p
    return inputs.ricker_problem(n, ts, seed=0, m_dtype=np.float32)


def cpu_baseline(prob, wl, budget_s=15.0):
    """FP64 oracle on the host cores, on a bounded sample: the workload's grid,
    a few of its time steps from the same start (steps scaled to the budget)."""
    import oracle
    threads = os.cpu_count() or 1
    n = wl["n"]
    m64 = prob.m.astype(np.float64)
    phi64 = prob.phi.astype(np.float64)
    hx = 1.0 / (n + 1)
    u0, u1 = oracle.adi_init(m64, phi64, hx, hx, prob.tau)
    wav = prob.wavelet.astype(np.float32).astype(np.float64) if prob.wavelet is not None else None
    t0 = time.perf_counter()
    up, uc, _ = oracle.adi_run(m64, u0, u1, hx, hx, prob.tau, 1, k0=1, src=prob.src, wavelet=wav,
                               threads=threads)
    t1 = time.perf_counter() - t0
    extra = int(max(0, min(wl["time_steps"] - 1, budget_s / max(t1, 1e-6) - 1)))
    steps = 1
    t_total = t1
    if extra > 0:
        t0 = time.perf_counter()
        oracle.adi_run(m64, up, uc, hx, hx, prob.tau, extra, k0=2, src=prob.src, wavelet=wav,
                       threads=threads)
        t_total += time.perf_counter() - t0
        steps += extra
    return {"value": float(n * n * steps / t_total), "unit": UNIT, "cores": threads,
            "kind": "oracle",
            "sample": "%d of the workload's %d ADI steps on the full %dx%d grid, FP64, %d threads"
                      % (steps, wl["time_steps"], n, n, threads)}


def run_reference(args, wl, rank):
    """The reference arm: the FP64 oracle as it stands, on the host cores."""
    if rank != 0:
        return None
    import oracle
    prob = make_problem(wl)
    threads = os.cpu_count() or 1
    n = wl["n"]
    m64 = prob.m.astype(np.float64)
    hx = 1.0 / (n + 1)
    u0, u1 = oracle.adi_init(m64, prob.phi.astype(np.float64), hx, hx, prob.tau)
    wav = prob.wavelet.astype(np.float32).astype(np.float64) if prob.wavelet is not None else None
    # each bench step: a bounded sample of the workload (ADI steps on the full grid)
    sample_steps = max(1, min(wl["time_steps"], int(2e8 // (n * n)) or 1))
    state = [u0, u1, 1]

    def one():
        up, uc, k = state
        up, uc, _ = oracle.adi_run(m64, up, uc, hx, hx, prob.tau, sample_steps, k0=k,
                                   src=prob.src, wavelet=wav, threads=threads)
        state[0], state[1], state[2] = up, uc, k + sample_steps

    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    val = n * n * sample_steps * args.steps / dt
    sample = ("%d ADI steps of the %dx%d grid per bench step (of the workload's %d), FP64, %d threads"
              % (sample_steps, n, n, wl["time_steps"], threads))
    return {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": args.workload, "n": n, "time_steps": wl["time_steps"]},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ricker_16384", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

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
        out = run_single(ctx)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _clock_sampler(ctx):
    vis = [v for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    lr = ctx["local_rank"]
    return ClockSampler(vis[lr].strip() if lr < len(vis) else lr)


def _timed(ctx, step_fn, launch_count):
    """Warm-up, then K steps between barriers + syncs, timed by CUDA events on
    the launching stream; returns (max_ms over ranks, own ms, launches, clocks)."""
    import torch
    args, world, rank, dist = ctx["args"], ctx["world"], ctx["rank"], ctx["dist"]
    stream = torch.cuda.current_stream()
    clocks = _clock_sampler(ctx)
    if rank == 0:
        clocks.start()
        time.sleep(0.5)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step_fn()
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = launch_count() - l0
    if world > 1:
        dist.barrier()
    clk = clocks.stop() if rank == 0 else None
    ms = ev0.elapsed_time(ev1)
    t = torch.tensor([ms], dtype=torch.float64, device=ctx["dev"])
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item()), ms, launches, clk


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


def run_single(ctx):
    import torch
    from paper_2006_10142_gb300 import api, autotune
    args, wl, world, rank, dev = ctx["args"], ctx["wl"], ctx["world"], ctx["rank"], ctx["dev"]
    n, ts = wl["n"], wl["time_steps"]
    prob = make_problem(wl)
    m_d = torch.from_numpy(prob.m).to(dev)
    phi_d = torch.from_numpy(prob.phi.astype(np.float32)).to(dev)
    src = prob.src
    wav_d = torch.from_numpy(prob.wavelet.astype(np.float32)).to(dev) if prob.wavelet is not None else None
    h = api.AdiWave(m_d, phi_d, prob.tau, src=src, wavelet=wav_d)
    tuned = None
    if not args.no_autotune:
        tuned = autotune.apply(h, steps=2, warmup=1)

    def bench_step():
        h.reset(phi_d)
        h.run(ts, src=src, wavelet=wav_d)

    for _ in range(max(args.warmup, 0)):
        bench_step()
    h.sync_status()
    h.profile(True)
    h.profile_read()
    max_ms, _, launches, clk = _timed(ctx, bench_step, h.launch_count)
    kms, kcnt = h.profile_read()
    h.profile(False)
    h.sync_status()
    value = world * n * n * ts * args.steps / (max_ms / 1e3)
    tun = h.tuning()
    # the kernels the plan launches: the TMA-pipelined forms (stage 3) or the
    # one-CTA-per-tile forms
    xname = "x_pipe_kernel" if tun.get("x_stage") == 3 else "x_sweep_kernel"
    yname = "y_pipe_kernel" if tun.get("y_stage") == 3 else "y_sweep_kernel"
    roof = _roofline(kms, kcnt, {0: xname, 1: yname},
                     {0: BYTES_X * n * n, 1: BYTES_Y * n * n}, args.workload)
    roof["step_gbs_32B"] = 32.0 * n * n * ts * args.steps / (max_ms / 1e3) / 1e9

    e2e = None
    if not args.no_e2e:
        m_h = torch.from_numpy(prob.m).pin_memory()
        phi_h = torch.from_numpy(prob.phi.astype(np.float32)).pin_memory()
        wav_h = (torch.from_numpy(prob.wavelet.astype(np.float32)).pin_memory()
                 if prob.wavelet is not None else None)
        out_h = torch.empty((n, n), dtype=torch.float32).pin_memory()
        # Each step uploads its inputs, runs and reads its result back.  The
        # copies run on their own streams: the upload of step i + 1 (into the
        # other of two device input sets) and the read-back of step i overlap
        # the compute of the neighbouring steps.
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
        e2e = {"value": world * n * n * ts * args.steps / e_dt, "unit": UNIT,
               "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(n * n * 4)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(prob, wl)
    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "time_steps": ts,
                       "medium": "seeded c-field 1 + 2 sigmoid(8 Gaussian bumps), m = c^2"
                       if wl["kind"] == "ricker" else "c = 1",
                       "source": "Ricker f=20" if wl["kind"] == "ricker" else "none",
                       "l2": "inputs larger than L2 (4 FP32 fields of %.0f MiB)" % (n * n * 4 / 2**20),
                       "timed_launches": "direct launches with per-kernel CUDA events",
                       "e2e_copies": "per step: H2D of m, phi, wavelet and D2H of u on two copy "
                                     "streams, overlapping the neighbouring steps' compute",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "tuning": h.tuning(), "autotuned": tuned is not None},
            "roofline": roof, "gpu_launches": int(launches), "clocks": clk, "e2e": e2e,
            "cpu_baseline": cpu,
        }
    h.close()
    return out


def run_batch(ctx):
    """64 shots with n from {256, 512, 1024, 2048}, one persistent launch per step;
    the plain kernels launched per shot are timed beside it for comparison."""
    import torch
    from paper_2006_10142_gb300 import api, inputs, shard
    args, wl, world, rank, dev = ctx["args"], ctx["wl"], ctx["world"], ctx["rank"], ctx["dev"]
    ts = wl["time_steps"]
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
    B.profile(True)
    B.profile_read()
    max_ms, _, launches, clk = _timed(ctx, bench_step, B.launch_count)
    kms, kcnt = B.profile_read()
    B.profile(False)
    B.sync_status()
    roof = _roofline(kms, kcnt, {2: "batch_step_kernel"}, {2: 32 * pts})
    # the plain single-grid kernels, one launch per shot and sweep, same work
    B.set_mode(1)
    for _ in range(2):
        bench_step()
    plain_ms, _, _, _ = _timed(ctx, bench_step, B.launch_count)
    B.set_mode(0)
    value = pts_all * ts * args.steps / (max_ms / 1e3)
    out = None
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": max_ms / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": args.workload, "shots": len(sizes_all),
                          "points_per_step": pts_all, "time_steps": ts,
                          "l2": "inputs larger than L2 (%.0f MiB per field over all shots)"
                          % (pts_all * 4 / 2**20),
                          "parallelism": "shot-sharded" if world > 1 else "single GPU",
                          "plain_per_shot_value": pts_all * ts * args.steps / (plain_ms / 1e3)},
               "roofline": roof, "gpu_launches": int(launches), "clocks": clk, "e2e": None,
               "cpu_baseline": None}
    B.close()
    return out


def run_adjoint(ctx):
    """1024^2, 64 receivers, 2000 steps, checkpoint every 50: time of the
    gradient (adjoint sweep with recomputation) per time step."""
    import torch
    from paper_2006_10142_gb300 import api, inputs
    args, wl, world, rank, dev = ctx["args"], ctx["wl"], ctx["world"], ctx["rank"], ctx["dev"]
    n, ts, every = wl["n"], wl["time_steps"], wl["ckpt_every"]
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
    f_ms, _, _, _ = _timed(ctx, forward, h.launch_count)
    forward()
    adj_ms, _, launches, clk = _timed(ctx, grad, h.launch_count)
    h.sync_status()
    out = None
    if rank == 0:
        per_step = adj_ms / args.steps / ts
        out = {"metric": "adjoint gradient time/step", "value": per_step, "unit": "ms",
               "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": adj_ms / args.steps, "higher_is_better": False,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32 (FP64 gradient)",
               "data": "synthetic",
               "config": {"workload": args.workload, "n": n, "time_steps": ts,
                          "receivers": wl["n_rec"], "ckpt_every": every,
                          "forward_ms_per_time_step": f_ms / args.steps / ts,
                          "adjoint_over_forward": (adj_ms / f_ms) if f_ms > 0 else None},
               "roofline": None, "gpu_launches": int(launches), "clocks": clk, "e2e": None,
               "cpu_baseline": None}
    h.close()
    return out


if __name__ == "__main__":
    main()
