"""Host logic of the shot-parallel multi-GPU path, on CPU with gloo ranks.

Two ranks each compute their share of a 64-shot batch; an all_gather checks
that the shares are disjoint, cover every shot, agree across ranks and are
balanced.  A max-reduction of per-rank timings (the benchmark's clock rule)
is checked the same way.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2006_10142_gb300 import inputs, shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = inputs.batch_sizes(64, seed=0)
    shapes = [(n, n) for n in sizes]
    mine = shard.local_shots(shapes, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((gathered, float(t.item())))
    dist.destroy_process_group()


def test_two_rank_partition_with_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(i for part in gathered for i in part)
    assert flat == list(range(64))
    assert not set(gathered[0]) & set(gathered[1])
    sizes = inputs.batch_sizes(64, seed=0)
    pts = [n * n for n in sizes]
    assert shard.imbalance(pts, world) < 1.05
    assert tmax == 2.0


def test_partition_edge_cases():
    assert shard.partition([], 3) == [[], [], []]
    assert shard.partition([5], 2) == [[0], []]
    assert shard.partition([4, 4, 4, 4], 4) == [[0], [1], [2], [3]]
    with pytest.raises(ValueError):
        shard.partition([1], 0)


# ---------------------------------------------------------------------------
# the sharded batch end to end: every rank advances its own shots (with the
# FP64 oracle standing in for the GPU, on CPU), rank 0 gathers the results and
# compares them, shot by shot, with one process that advanced every shot
# ---------------------------------------------------------------------------
SMALL_SIZES = [24, 40, 16, 33, 48, 20, 29]
SMALL_STEPS = 6


def _advance_shot(b):
    import numpy as np
    import oracle
    n = SMALL_SIZES[b]
    p = inputs.ricker_problem(n, SMALL_STEPS, seed=b, m_dtype=np.float32)
    h = 1.0 / (n + 1)
    m64 = p.m.astype(np.float64)
    u0, u1 = oracle.adi_init(m64, p.phi.astype(np.float64), h, h, p.tau)
    wav = 1e3 * p.wavelet.astype(np.float64)   # a visible field after a few steps
    _, uc, _ = oracle.adi_run(m64, u0, u1, h, h, p.tau, SMALL_STEPS, src=p.src, wavelet=wav)
    return uc


def _batch_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.local_shots([(n, n) for n in SMALL_SIZES], rank, world)
    out = {b: _advance_shot(b) for b in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, out)
    if rank == 0:
        q.put(gathered)
    dist.destroy_process_group()


def test_two_rank_sharded_batch_matches_one_process():
    import numpy as np
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    merged = {}
    for part in gathered:
        assert not set(part) & set(merged)      # every shot advanced by one rank only
        merged.update(part)
    assert sorted(merged) == list(range(len(SMALL_SIZES)))
    for b in range(len(SMALL_SIZES)):
        ref = _advance_shot(b)
        assert merged[b].shape == (SMALL_SIZES[b], SMALL_SIZES[b])
        assert np.array_equal(merged[b], ref)
        assert np.abs(ref).max() > 0
