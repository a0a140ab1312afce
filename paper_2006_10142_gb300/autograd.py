"""torch.autograd.Function over the C ABI: forward = adi_wave_run with receivers,
backward = adi_wave_adjoint.

    traces = simulate(m, wavelet, src=(ix, iy), rec=rec, steps=S, dt=tau)
    loss = 0.5 * ((traces - data) ** 2).sum()
    loss.backward()          # m.grad = dJ/dm (m = c^2), wavelet.grad = dJ/dw

m is the coefficient of the Laplacian (c^2).  If m is built from a speed
tensor c in torch (m = c * c), autograd applies dJ/dc = 2c dJ/dm itself.  The
library sums the gradient wrt m in FP32 within a checkpoint segment and in
FP64 across segments, and returns it in m's dtype (FP32).  Checkpoints of the forward run are kept every `ckpt_every`
steps and the reverse sweep recomputes between them.
"""
from __future__ import annotations

from typing import Optional, Sequence, Tuple

import torch

from .api import AdiWave


class _Simulate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, wavelet, phi, dt, src, rec, steps, ckpt_every, lx, ly, start):
        h = AdiWave(m.detach(), phi.detach(), dt, lx=lx, ly=ly, start=start, src=src,
                    wavelet=wavelet.detach())
        h.set_checkpointing(ckpt_every)
        traces = h.run(steps, src=src, wavelet=wavelet.detach(), rec=rec)
        ctx.h = h
        return traces

    @staticmethod
    def backward(ctx, grad_traces):
        h = ctx.h
        gm, gw = h.adjoint(grad_traces.detach().float().contiguous())
        h.close()
        ctx.h = None
        return (gm.to(torch.float32), gw, None, None, None, None, None, None, None, None, None)


def simulate(m: torch.Tensor, wavelet: torch.Tensor, src: Tuple[int, int],
             rec: Sequence[Sequence[int]], steps: int, dt: float,
             phi: Optional[torch.Tensor] = None, ckpt_every: int = 50, lx: float = 1.0,
             ly: float = 1.0, start: str = "paper") -> torch.Tensor:
    """Receiver traces [steps, n_rec] of the ADI run; differentiable in m and wavelet."""
    if phi is None:
        phi = torch.zeros_like(m)
    return _Simulate.apply(m, wavelet, phi, float(dt), tuple(src), rec, int(steps),
                           int(ckpt_every), float(lx), float(ly), start)
