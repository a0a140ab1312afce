"""Shot-parallel misfit gradient with a shared medium (full-waveform
inversion's inner step).

Many shots (source positions and their recorded traces) see the same medium
m = c^2.  The misfit is J = sum over shots of 1/2 sum_{s,r} (u_shot^{k0+s+1}(rec r)
- d_shot[s][r])^2 and its gradient the sum of the shots' gradients.  Each rank
(one process per GPU) owns a subset of the shots (shard.partition, balanced
by grid points), runs every owned shot forward with its receivers and then
its adjoint (adi_wave_adjoint: the transposed sweeps backward in time with
checkpointing), and adds the shot gradients; one all-reduce then sums the
ranks' gradients and misfits.  The paper's conclusion points to clusters of
GPUs as the way to scale the method; shots are the natural unit, since a
single grid does not split without an exchange in every sweep.

The per-shot work is a callable, so the reduction logic is the same whatever
computes a shot (the default runs the CUDA library on the current device).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np

from . import shard


@dataclass
class Shot:
    """One shot: point source, wavelet samples w(t_k), receivers and the
    observed traces d[s][r] (same layout as adi_wave_run's traces)."""
    src: Tuple[int, int]
    wavelet: object          # device float32 tensor (GPU path) or array
    rec: np.ndarray          # [n_rec, 2] int32 (ix, iy)
    data: object             # [steps, n_rec] observed traces


def gpu_shot_gradient(m, shot: Shot, tau: float, steps: int, every: int):
    """(J_shot, dJ/dm as a float64 device tensor) of one shot from rest, on
    the current CUDA device, through the library's forward run and adjoint."""
    import torch

    from . import api
    h = api.AdiWave(m, torch.zeros_like(m), tau, src=shot.src, wavelet=shot.wavelet)
    try:
        h.set_checkpointing(every)
        tr = h.run(steps, src=shot.src, wavelet=shot.wavelet, rec=shot.rec)
        resid = tr - shot.data
        gm, _ = h.adjoint(resid, ckpt_every=every)
        h.sync_status()
        J = 0.5 * float((resid.double() ** 2).sum())
        return J, gm
    finally:
        h.close()


def shot_points(shots: Sequence[Shot], shape: Tuple[int, int]) -> List[int]:
    """Work per shot (grid points per step): every shot shares the grid."""
    return [shape[0] * shape[1]] * len(shots)


def misfit_gradient(m, shots: Sequence[Shot], tau: float, steps: int, every: int = 50,
                    shot_gradient: Optional[Callable] = None, group=None):
    """Misfit and gradient wrt m summed over all shots and all ranks.

    Each rank computes the shots that shard.partition gives it; with
    torch.distributed initialised (world > 1) the per-rank sums are added by
    one all-reduce over `group` (NCCL for CUDA tensors).  Returns
    (J, dJ/dm) with dJ/dm a float64 tensor of m's shape on m's device."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_available() and dist.is_initialized() else 1
    rank = dist.get_rank(group) if world > 1 else 0
    fn = shot_gradient or gpu_shot_gradient
    ny, nx = tuple(m.shape)
    mine = shard.partition(shot_points(shots, (nx, ny)), world)[rank]
    g = torch.zeros((ny, nx), dtype=torch.float64, device=m.device)
    J = torch.zeros((1,), dtype=torch.float64, device=m.device)
    for s in mine:
        Js, gs = fn(m, shots[s], tau, steps, every)
        g += torch.as_tensor(gs, dtype=torch.float64, device=m.device)
        J += float(Js)
    if world > 1:
        dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(J, op=dist.ReduceOp.SUM, group=group)
    return float(J.item()), g


def gradient_wrt_speed(grad_m, c):
    """dJ/dc = 2 c dJ/dm (m = c^2)."""
    return 2.0 * c * grad_m
