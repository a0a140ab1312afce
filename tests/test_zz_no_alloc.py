"""adi_wave_step_noalloc (a library call with no counterpart in the paper)
against the handle API's adi_wave_step on the same grid and state.

Both run the same x and y sweep kernels with the same launch plan, so the
states after each step must agree bit for bit; calls that alternate between
two grids check that the static scratch and grid record are reused
correctly.  The file sorts
last so that the calls also run after every other test has used the library.
"""
import math

import numpy as np
import pytest
import torch

from paper_2006_10142_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu


def _pitched(a, ld, dev):
    ny, nx = a.shape
    out = torch.zeros((ny, ld), dtype=torch.float32, device=dev)
    out[:, :nx] = torch.as_tensor(a, dtype=torch.float32, device=dev)
    return out


def _case(nx, ny, extra_pitch, seed, dev):
    """A handle on an nx x ny grid and the same state in caller-owned pitched
    buffers (row pitch roundup(nx, 32) + extra_pitch, padding zero)."""
    m = inputs.m_field(nx, ny, seed, dtype=np.float32)
    h = min(1.0 / (nx + 1), 1.0 / (ny + 1))
    tau = 0.5 * h / math.sqrt(float(m.max()))
    phi = inputs.m_field(nx, ny, seed + 1, dtype=np.float32) * np.float32(1e-3)
    src = (nx // 3, ny // 2)
    wav = torch.from_numpy(inputs.wavelet_samples(8, tau).astype(np.float32)).to(dev)
    sim = api.AdiWave(torch.from_numpy(m).to(dev), torch.from_numpy(phi).to(dev), tau, src=src,
                      wavelet=wav)
    up, uc, k = sim.state()
    assert k == 1
    ld = (nx + 31) // 32 * 32 + extra_pitch
    return dict(nx=nx, ny=ny, ld=ld, tau=tau, m_max=float(m.max()), src=src, wav=wav, sim=sim,
                m=_pitched(m, ld, dev), a=_pitched(up.cpu().numpy(), ld, dev),
                b=_pitched(uc.cpu().numpy(), ld, dev), k=k)


def test_noalloc_matches_handle_step_alternating_grids():
    """Two calls on each of two grids, alternating, so that every call finds
    the static array holding the other grid's w: a 300 x 200 grid and a
    1100 x 1030 grid with a row pitch 32 floats wider than needed, whose
    default plan runs both TMA-pipelined sweeps (x_stage = y_stage = 3)."""
    dev = torch.device("cuda:0")
    cases = [_case(300, 200, 0, 3, dev), _case(1100, 1030, 32, 5, dev)]
    tun = cases[1]["sim"].tuning()
    assert tun["x_stage"] == 3 and tun["y_stage"] == 3, tun
    for step in range(2):
        for c in cases:
            c["sim"].step(src=c["src"], wavelet=c["wav"])
            api.step_noalloc(c["m"], c["b"], c["a"], c["nx"], c["tau"], c["m_max"], c["k"] + step,
                             src=c["src"], wavelet=c["wav"])
            c["a"], c["b"] = c["b"], c["a"]          # b now holds u^{k+step+1}
        torch.cuda.synchronize()
        for c in cases:
            _, ref, kk = c["sim"].state()
            assert kk == c["k"] + step + 1
            got = c["b"][:, :c["nx"]]
            assert torch.equal(got, ref), float((got - ref).abs().max())
            assert torch.count_nonzero(c["b"][:, c["nx"]:]) == 0   # padding stays zero
            assert float(ref.abs().max()) > 0
    for c in cases:
        c["sim"].close()


def test_noalloc_rejects_grid_beyond_static_scratch():
    dev = torch.device("cuda:0")
    nx, ny, ld = 2048, 2049, 2048      # ld * ny = 4196352 > 4194304
    z = torch.zeros((ny, ld), dtype=torch.float32, device=dev)
    u = torch.zeros_like(z)
    m = torch.ones_like(z)
    with pytest.raises(_lib.AdiError) as ei:
        api.step_noalloc(m, z, u, nx, 1e-4, 1.0, 1)
    assert ei.value.code == _lib.ADI_EINVAL
    assert "at most 4194304" in str(ei.value)
