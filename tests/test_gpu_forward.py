"""GPU parity of the forward ADI path (C ABI) against the FP64 oracle.

Bar: relative L2 <= 1e-4 per field after the run (FP32 GPU vs FP64 oracle on
the same FP32-rounded inputs).  Grids cover one and several tiles per line,
ragged tails (sizes that are not multiples of the chunk, the strip width or
a power of two), degenerate 1-wide grids, non-square grids, every chunk
length and CR-to-PCR switch size, the cluster path of the y sweep, the FP64
fallback, the Taylor start, receivers and graph replay.
"""
import math

import numpy as np
import pytest

from paper_2006_10142_gb300 import inputs
from helpers import gpu_run, oracle_run, rel_l2, smooth_state

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _problem(nx, ny, steps, seed=0, cfl=0.5, with_src=True):
    m = inputs.m_field(nx, ny, seed)
    h = min(1.0 / (nx + 1), 1.0 / (ny + 1))
    tau = cfl * h / math.sqrt(m.max())
    phi = smooth_state(nx, ny, seed, 1e-2)
    src = (nx // 3, (2 * ny) // 3) if with_src else None
    wav = inputs.wavelet_samples(steps + 2, tau, fp=3.0) if with_src else None
    return m, phi, tau, src, wav


def test_standing_wave_128_closed_form():
    prob = inputs.standing_wave_problem(128, 200)
    g = gpu_run(prob.m, prob.phi, prob.tau, prob.steps)
    o = oracle_run(prob.m, prob.phi, prob.tau, prob.steps)
    assert g["k"] == 201
    e_prev = rel_l2(g["u_prev"], o["u_prev"])
    e_cur = rel_l2(g["u_cur"], o["u_cur"])
    assert e_prev < TOL and e_cur < TOL, (e_prev, e_cur)
    # exact discrete solution of the (1,1) mode: v^K = cos((K - 1/2) th) / cos(th / 2)
    n, tau = 128, prob.tau
    h = 1.0 / (n + 1)
    P = 4.0 / h ** 2 * math.sin(math.pi * h / 2) ** 2
    s = tau * tau / 2
    th = math.acos(1 - tau * tau * 2 * P / (2 * (1 + s * P) ** 2))
    K = 201
    amp = math.cos((K - 0.5) * th) / math.cos(th / 2)
    assert rel_l2(g["u_cur"], amp * prob.phi) < TOL


@pytest.mark.parametrize("nx,ny", [(37, 53), (1, 17), (17, 1), (1, 1), (100, 3), (129, 257),
                                   (300, 40), (513, 200), (1000, 700)])
def test_ragged_grids_match_oracle(nx, ny):
    steps = 12
    m, phi, tau, src, wav = _problem(nx, ny, steps, seed=nx + ny)
    rec = np.array([[i % nx, (3 * i) % ny] for i in range(5)], dtype=np.int32)
    g = gpu_run(m, phi, tau, steps, src=src, wavelet=wav, rec=rec)
    o = oracle_run(m, phi, tau, steps, src=src, wavelet=wav, rec=rec)
    assert rel_l2(g["u_cur"], o["u_cur"]) < TOL
    assert rel_l2(g["u_prev"], o["u_prev"]) < TOL
    assert rel_l2(g["traces"], o["traces"]) < TOL


@pytest.mark.parametrize("solver", [1, 2])
@pytest.mark.parametrize("kx,ky,pcr,W", [(4, 4, 32, 8), (8, 8, 2, 16), (16, 16, 8, 32),
                                         (32, 32, 32, 8), (16, 4, 16, 4), (4, 32, 4, 32)])
def test_tuning_variants_match_oracle(kx, ky, pcr, W, solver):
    nx, ny, steps = 300, 260, 8
    m, phi, tau, src, wav = _problem(nx, ny, steps, seed=7)
    tun = dict(chunk_x=kx, chunk_y=ky, pcr_size=pcr, cols_per_cta=W, solver=solver)
    g = gpu_run(m, phi, tau, steps, src=src, wavelet=wav, tuning=tun)
    o = oracle_run(m, phi, tau, steps, src=src, wavelet=wav)
    assert g["tuning"]["chunk_x"] == kx and g["tuning"]["chunk_y"] == ky
    assert rel_l2(g["u_cur"], o["u_cur"]) < TOL


@pytest.mark.parametrize("ny,ky,solver", [(4096, 4, 2), (8191, 4, 2), (3000, 8, 2),
                                          (4096, 8, 1), (8191, 16, 1), (3000, 8, 1),
                                          (16384, 16, 1)])
def test_cluster_y_sweep_matches_oracle(ny, ky, solver):
    """Columns long enough that the y sweep spans a thread-block cluster (DSMEM)."""
    nx, steps = 40, 6
    m, phi, tau, src, wav = _problem(nx, ny, steps, seed=3)
    g = gpu_run(m, phi, tau, steps, src=src, wavelet=wav, tuning=dict(chunk_y=ky, solver=solver))
    o = oracle_run(m, phi, tau, steps, src=src, wavelet=wav)
    assert rel_l2(g["u_cur"], o["u_cur"]) < TOL


def test_long_rows_single_cta():
    nx, ny, steps = 16384, 24, 4
    m, phi, tau, src, wav = _problem(nx, ny, steps, seed=4)
    g = gpu_run(m, phi, tau, steps, src=src, wavelet=wav)
    o = oracle_run(m, phi, tau, steps, src=src, wavelet=wav)
    assert rel_l2(g["u_cur"], o["u_cur"]) < TOL


def test_graph_replay_equals_direct_launches():
    nx, ny, steps = 200, 180, 10
    m, phi, tau, src, wav = _problem(nx, ny, steps, seed=11)
    a = gpu_run(m, phi, tau, steps, src=src, wavelet=wav, tuning=dict(use_graph=1))
    b = gpu_run(m, phi, tau, steps, src=src, wavelet=wav, tuning=dict(use_graph=-1))
    np.testing.assert_array_equal(a["u_cur"], b["u_cur"])
    np.testing.assert_array_equal(a["u_prev"], b["u_prev"])


def test_taylor_start_and_velocity():
    nx, ny, steps = 64, 48, 30
    m, phi, tau, src, wav = _problem(nx, ny, steps, seed=2)
    psi = smooth_state(nx, ny, 9, 1e-2)
    g = gpu_run(m, phi, tau, steps, psi=psi, src=src, wavelet=wav, start="taylor2")
    o = oracle_run(m, phi, tau, steps, psi=psi, src=src, wavelet=wav, start="taylor2")
    assert rel_l2(g["u_cur"], o["u_cur"]) < TOL


def test_non_unit_domain():
    nx, ny, steps = 90, 70, 15
    m, phi, tau, src, wav = _problem(nx, ny, steps, seed=5)
    g = gpu_run(m, phi, tau * 2, steps, src=src, wavelet=wav, lx=2.0, ly=1.5)
    o = oracle_run(m, phi, tau * 2, steps, src=src, wavelet=wav, lx=2.0, ly=1.5)
    assert rel_l2(g["u_cur"], o["u_cur"]) < TOL


@pytest.mark.parametrize("nx,ny", [(120, 90), (600, 70)])
@pytest.mark.parametrize("fp64", ["auto", "always"])
def test_fp64_fallback_weak_dominance(fp64, nx, ny):
    """tau = 5h: (|a| + |c|)/|b| = 2s/(1 + 2s) > 0.9, the FP64 elimination path
    (rows of 120: K = 8; rows of 600: K = 16)."""
    steps = 10
    h = 1.0 / (nx + 1)
    m = np.ones((ny, nx))
    phi = smooth_state(nx, ny, 1)
    tau = 5 * h
    g = gpu_run(m, phi, tau, steps, fp64=fp64)
    assert g["tuning"]["chunk_x"] == (16 if nx >= 512 else 8)
    o = oracle_run(m, phi, tau, steps)
    assert rel_l2(g["u_cur"], o["u_cur"]) < TOL


@pytest.mark.parametrize("nx,ny,scale2", [(300, 260, 1.3), (1000, 700, 1.0), (120, 90, 60.0)])
def test_reset_with_new_medium_matches_oracle(nx, ny, scale2):
    """Run, then restart the same handle with another medium and initial field
    (Eq. CN2 again) and run on: the captured step graphs are kept when the new
    medium gives the same launch plan and rebuilt when it does not (scale 60
    makes the systems weakly dominant, which switches to FP64 elimination)."""
    import torch
    from paper_2006_10142_gb300 import api
    from helpers import f32
    steps = 12
    m1, phi1, tau, src, wav = _problem(nx, ny, steps, seed=5)
    m2 = scale2 * inputs.m_field(nx, ny, 6)
    phi2 = smooth_state(nx, ny, 7, 1e-2)
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(f32(a)).to(dev)
    wav_t = t(wav)
    h = api.AdiWave(t(m1), t(phi1), tau, src=src, wavelet=wav_t)
    h.run(steps, src=src, wavelet=wav_t)
    h.run(steps, src=src, wavelet=wav_t)  # graph replay on the first medium
    h.reset(t(phi2), m=t(m2), src=src, wavelet=wav_t)
    h.run(steps, src=src, wavelet=wav_t)
    up, uc, k = h.state()
    h.sync_status()
    h.close()
    assert k == steps + 1
    o = oracle_run(m2, phi2, tau, steps, src=src, wavelet=wav)
    assert rel_l2(uc.double().cpu().numpy(), o["u_cur"]) < TOL
    assert rel_l2(up.double().cpu().numpy(), o["u_prev"]) < TOL


def test_state_roundtrip_and_levels():
    import torch
    from paper_2006_10142_gb300 import api
    nx, ny = 50, 40
    m, phi, tau, src, wav = _problem(nx, ny, 5, seed=1)
    dev = torch.device("cuda:0")
    h = api.AdiWave(torch.tensor(m, dtype=torch.float32, device=dev),
                    torch.tensor(phi, dtype=torch.float32, device=dev), tau)
    up, uc, k = h.state()
    assert k == 1
    np.testing.assert_array_equal(up.cpu().numpy(), phi.astype(np.float32))
    h.run(3)
    _, _, k = h.state()
    assert k == 4
    a = torch.randn(ny, nx, device=dev)
    b = torch.randn(ny, nx, device=dev)
    h.set_state(a, b, 17)
    up, uc, k = h.state()
    assert k == 17 and torch.equal(up, a) and torch.equal(uc, b)
    h.step()
    _, _, k = h.state()
    assert k == 18
    h.close()


def test_non_finite_state_sets_numeric_flag():
    import torch
    from paper_2006_10142_gb300 import api
    nx, ny = 33, 21
    dev = torch.device("cuda:0")
    h = api.AdiWave(torch.ones(ny, nx, device=dev), torch.zeros(ny, nx, device=dev), 0.01)
    bad = torch.zeros(ny, nx, device=dev)
    bad[3, 4] = float("nan")
    h.set_state(bad, bad, 1)
    h.step()
    with pytest.raises(api.AdiError) as ei:
        h.sync_status()
    assert ei.value.code == 4
    h.sync_status()  # the word was cleared
    h.close()


@pytest.mark.parametrize("bad", [0.0, -1.0, float("nan"), float("inf")])
def test_medium_must_be_finite_and_positive(bad):
    """The range scan of m (Eq. f1 needs c^2 > 0) rejects a zero, negative or
    non-finite coefficient anywhere, at init and at a reset with a new
    medium; a rejected reset leaves the handle's medium and state as they
    were."""
    import torch
    from helpers import f32
    from paper_2006_10142_gb300 import _lib, api
    dev = torch.device("cuda:0")
    nx, ny, steps = 70, 45, 5
    m, phi, tau, src, wav = _problem(nx, ny, steps, seed=11)
    m_d = torch.from_numpy(f32(m)).to(dev)
    phi_d = torch.from_numpy(f32(phi)).to(dev)
    mb = m_d.clone()
    mb[ny // 2, nx - 1] = bad
    with pytest.raises(_lib.AdiError) as ei:
        api.AdiWave(mb, phi_d, tau)
    assert ei.value.code == _lib.ADI_EINVAL
    h = api.AdiWave(m_d, phi_d, tau)
    with pytest.raises(_lib.AdiError) as ei:
        h.reset(phi_d, m=mb)
    assert ei.value.code == _lib.ADI_EINVAL
    h.run(steps, src=src, wavelet=torch.from_numpy(f32(wav)).to(dev))
    h.sync_status()
    up, uc, k = h.state()
    h.close()
    o = oracle_run(m, phi, tau, steps, src=src, wavelet=wav)
    assert k == steps + 1
    assert rel_l2(uc.double().cpu().numpy(), o["u_cur"]) < TOL
    assert rel_l2(up.double().cpu().numpy(), o["u_prev"]) < TOL


def test_invalid_run_arguments():
    import torch
    from paper_2006_10142_gb300 import api
    dev = torch.device("cuda:0")
    h = api.AdiWave(torch.ones(10, 12, device=dev), torch.zeros(10, 12, device=dev), 0.01)
    with pytest.raises(api.AdiError):
        h.run(3, src=(12, 0), wavelet=torch.zeros(5, device=dev))
    with pytest.raises(api.AdiError):
        h.run(3, rec=[[0, 10]])
    with pytest.raises(api.AdiError):
        h.set_tuning(chunk_x=5)
    h.close()
    with pytest.raises(api.AdiError):
        api.AdiWave(-torch.ones(10, 12, device=dev), torch.zeros(10, 12, device=dev), 0.01)


@pytest.mark.parametrize("nx,ny", [(1000, 700), (8200, 40), (40, 5000), (333, 2049)])
@pytest.mark.parametrize("xs,ys", [(1, 1), (2, 2), (3, 3), (2, 3), (3, 1)])
def test_staging_modes_match_oracle(nx, ny, xs, ys):
    """Every way the sweeps fetch their operands (shared-memory staging, direct
    or L2-prefetched loads, the TMA-pipelined persistent kernels) on ragged
    grids: a partial last row block, rows split over two TMA boxes, a strip
    past nx, cluster ranks whose boxes lie wholly beyond ny."""
    from paper_2006_10142_gb300 import _lib
    steps = 6
    m, phi, tau, src, wav = _problem(nx, ny, steps, seed=nx + 3 * ny)
    tun = dict(x_stage=xs, y_stage=ys, cols_per_cta=16, chunk_y=32, cta_threads_y=512)
    try:
        g = gpu_run(m, phi, tau, steps, src=src, wavelet=wav, tuning=tun)
    except _lib.AdiError as e:
        assert e.code == _lib.ADI_EUNSUPPORTED, str(e)
        pytest.skip("shape not supported by this staging mode: %s" % e)
    assert g["tuning"]["x_stage"] == xs and g["tuning"]["y_stage"] == ys
    o = oracle_run(m, phi, tau, steps, src=src, wavelet=wav)
    assert rel_l2(g["u_cur"], o["u_cur"]) < TOL
    assert rel_l2(g["u_prev"], o["u_prev"]) < TOL


@pytest.mark.parametrize("nx,ny", [(16384, 9), (12000, 33), (9000, 20), (2500, 40)])
@pytest.mark.parametrize("xc", [1, 2, 4])
def test_row_split_over_cta_pair_matches_oracle(nx, ny, xc):
    """Rows solved by one CTA or split over a cluster of two or four (the
    parts meet through DSMEM), including rows whose last parts are mostly or
    wholly padding."""
    steps = 4
    m, phi, tau, src, wav = _problem(nx, ny, steps, seed=nx % 97 + ny)
    tun = dict(x_stage=3, chunk_x=32, x_cluster=xc, rows_per_cta=1)
    g = gpu_run(m, phi, tau, steps, src=src, wavelet=wav, tuning=tun)
    assert g["tuning"]["x_cluster"] == xc
    o = oracle_run(m, phi, tau, steps, src=src, wavelet=wav)
    assert rel_l2(g["u_cur"], o["u_cur"]) < TOL
    assert rel_l2(g["u_prev"], o["u_prev"]) < TOL


@pytest.mark.parametrize("nx,ny,W,ky,ty", [(40, 5000, 16, 32, 256), (300, 1500, 16, 32, 512),
                                           (1100, 9000, 16, 32, 256), (77, 16384, 16, 32, 256),
                                           (33, 32768, 16, 32, 512), (50, 2049, 16, 16, 512),
                                           (17, 64, 16, 32, 256), (100, 5000, 32, 32, 512),
                                           (1100, 16384, 32, 32, 512), (70, 3000, 32, 16, 512)])
def test_y_segments_through_global_memory_match_oracle(nx, ny, W, ky, ty):
    """The y sweep without clusters (y_stage 4): persistent co-resident CTAs
    whose column segments meet through global memory; strips of 16 and 32
    columns, one segment per column (17 x 64), up to 32 segments (16384 rows
    at 512 per segment, 32768 at 1024), partial last segments and strips past
    nx; the run replays step pairs from a CUDA graph."""
    steps = 6
    m, phi, tau, src, wav = _problem(nx, ny, steps, seed=nx + ny)
    tun = dict(y_stage=4, chunk_y=ky, cta_threads_y=ty, cols_per_cta=W)
    g = gpu_run(m, phi, tau, steps, src=src, wavelet=wav, tuning=tun)
    assert g["tuning"]["y_stage"] == 4 and g["tuning"]["chunk_y"] == ky
    assert g["tuning"]["cols_per_cta"] == W
    o = oracle_run(m, phi, tau, steps, src=src, wavelet=wav)
    assert rel_l2(g["u_cur"], o["u_cur"]) < TOL
    assert rel_l2(g["u_prev"], o["u_prev"]) < TOL


@pytest.mark.parametrize("nx,ny", [(16384, 600), (12000, 33), (9000, 20), (4096, 300),
                                   (2500, 1000)])
@pytest.mark.parametrize("xc", [2, 4, 8])
@pytest.mark.parametrize("kx", [32, 16])
def test_x_band_form_matches_oracle(nx, ny, xc, kx):
    """The band form of the x sweep (x_stage 5): clusters of 2, 4 or 8 CTAs
    walk bands of consecutive rows with rows j - 1, j, j + 1 of u^k in a
    shared-memory ring; bands of one to many rows, the grid's first and last
    rows (zero halo rows from the copies' fill), cluster ranks partly or
    wholly past the row; 32 or 16 unknowns per thread."""
    from paper_2006_10142_gb300 import _lib
    steps = 4
    m, phi, tau, src, wav = _problem(nx, ny, steps, seed=nx % 89 + ny)
    tun = dict(x_stage=5, chunk_x=kx, x_cluster=xc, rows_per_cta=1)
    try:
        g = gpu_run(m, phi, tau, steps, src=src, wavelet=wav, tuning=tun)
    except _lib.AdiError as e:
        assert e.code == _lib.ADI_EUNSUPPORTED, str(e)
        pytest.skip("shape not supported by the band form: %s" % e)
    assert g["tuning"]["x_stage"] == 5 and g["tuning"]["x_cluster"] == xc
    o = oracle_run(m, phi, tau, steps, src=src, wavelet=wav)
    assert rel_l2(g["u_cur"], o["u_cur"]) < TOL
    assert rel_l2(g["u_prev"], o["u_prev"]) < TOL
