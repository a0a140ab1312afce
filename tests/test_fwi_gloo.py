"""Shot-parallel misfit gradient with a shared medium (fwi.misfit_gradient)
on two gloo ranks on CPU: each rank computes its shots with the FP64 oracle
standing in for the GPU, one all-reduce adds the ranks' gradients and
misfits, and the result equals one process's sum over every shot."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2006_10142_gb300 import fwi, inputs

NX, NY, STEPS, N_SHOTS = 22, 18, 30, 5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _setup():
    m = inputs.m_field(NX, NY, 1)
    m_true = m * (1.0 + 0.05 * inputs.bump(NX, NY, 0.5, 0.5, 0.2))
    h = min(1.0 / (NX + 1), 1.0 / (NY + 1))
    tau = 1.5 * h / np.sqrt(m.max())
    wav = inputs.ricker(np.arange(STEPS + 2) * tau, fp=4.0, t0=0.05)
    rec = np.array([[i, 2] for i in range(1, NX - 1, 3)], dtype=np.int32)
    shots = []
    for s in range(N_SHOTS):
        src = (2 + 4 * s, NY - 3)
        d = _traces(m_true, tau, src, wav, rec)
        shots.append(fwi.Shot(src=src, wavelet=wav, rec=rec, data=d))
    return m, tau, shots


def _traces(m, tau, src, wav, rec):
    import oracle
    hx, hy = 1.0 / (NX + 1), 1.0 / (NY + 1)
    z = np.zeros((NY, NX))
    _, _, tr = oracle.adi_run(np.asarray(m, dtype=np.float64), z, z, hx, hy, tau, STEPS, src=src,
                              wavelet=wav, rec=rec)
    return tr


def oracle_shot_gradient(m, shot, tau, steps, every):
    import oracle
    mm = m.detach().cpu().numpy().astype(np.float64)
    hx, hy = 1.0 / (NX + 1), 1.0 / (NY + 1)
    tr = _traces(mm, tau, shot.src, shot.wavelet, shot.rec)
    resid = tr - shot.data
    z = np.zeros((NY, NX))
    g = oracle.adi_adjoint(mm, z, z, hx, hy, tau, steps, resid, shot.rec, src=shot.src,
                           wavelet=shot.wavelet)["grad_m"]
    return 0.5 * float(np.sum(resid ** 2)), g


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, tau, shots = _setup()
    J, g = fwi.misfit_gradient(torch.from_numpy(m), shots, tau, STEPS, 10,
                               shot_gradient=oracle_shot_gradient)
    if rank == 0:
        q.put((J, g.numpy()))
    dist.destroy_process_group()


def test_two_rank_gradient_allreduce_equals_one_process_sum():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    J2, g2 = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    m, tau, shots = _setup()
    J1, g1 = 0.0, np.zeros((NY, NX))
    for s in shots:
        Js, gs = oracle_shot_gradient(torch.from_numpy(m), s, tau, STEPS, 10)
        J1 += Js
        g1 += gs
    assert J1 > 0 and np.linalg.norm(g1) > 0
    assert abs(J2 - J1) <= 1e-12 * J1
    np.testing.assert_allclose(g2, g1, rtol=1e-12, atol=1e-12 * np.abs(g1).max())
    # one shard alone is not the whole gradient
    part = fwi.shard.partition(fwi.shot_points(shots, (NX, NY)), 2)
    assert all(len(p) > 0 for p in part)
