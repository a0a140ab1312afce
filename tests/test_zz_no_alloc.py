"""adi_wave_step_noalloc (a library call with no counterpart in the paper)
against the handle API's adi_wave_step on the same grid and state.

Both run the same x and y sweep kernels with the same launch plan, so the
states after each step must agree bit for bit; two calls in a row check that
the static scratch and grid record are reused correctly.  The file sorts
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


@pytest.mark.parametrize("nx,ny", [(300, 200), (1000, 1030)])
def test_noalloc_matches_handle_step_two_calls(nx, ny):
    dev = torch.device("cuda:0")
    m = inputs.m_field(nx, ny, 3, dtype=np.float32)
    h = min(1.0 / (nx + 1), 1.0 / (ny + 1))
    tau = 0.5 * h / math.sqrt(float(m.max()))
    phi = inputs.m_field(nx, ny, 4, dtype=np.float32) * np.float32(1e-3)
    src = (nx // 3, ny // 2)
    wav = torch.from_numpy(inputs.wavelet_samples(8, tau).astype(np.float32)).to(dev)
    m_d = torch.from_numpy(m).to(dev)
    sim = api.AdiWave(m_d, torch.from_numpy(phi).to(dev), tau, src=src, wavelet=wav)
    up, uc, k = sim.state()
    assert k == 1
    ld = (nx + 31) // 32 * 32
    m_p = _pitched(m, ld, dev)
    a = _pitched(up.cpu().numpy(), ld, dev)   # u^{k-1}
    b = _pitched(uc.cpu().numpy(), ld, dev)   # u^k
    for step in range(2):
        sim.step(src=src, wavelet=wav)
        api.step_noalloc(m_p, b, a, nx, tau, float(m.max()), k + step, src=src, wavelet=wav)
        a, b = b, a                            # b now holds u^{k+step+1}
        _, ref, kk = sim.state()
        torch.cuda.synchronize()
        assert kk == k + step + 1
        got = b[:, :nx]
        assert torch.equal(got, ref), float((got - ref).abs().max())
        assert torch.count_nonzero(b[:, nx:]) == 0   # padding stays zero
        assert float(ref.abs().max()) > 0
    sim.close()


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
