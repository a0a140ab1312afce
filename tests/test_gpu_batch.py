"""The batched form: many grids of uneven size, one persistent launch per step.

Every shot is checked against the FP64 oracle (relative L2 <= 1e-4); the
persistent kernel is checked against the plain kernels launched per shot; the
bounded dependency wait is made to run out on purpose (a wait target nothing
reaches) and must end with ADI_ETIMEOUT while the context stays usable.
"""
import math

import numpy as np
import pytest

from paper_2006_10142_gb300 import inputs
from helpers import f32, oracle_run, rel_l2, smooth_state

pytestmark = pytest.mark.gpu


def _shots(shapes, steps, seed0=0):
    out = []
    for b, (nx, ny) in enumerate(shapes):
        m = inputs.m_field(nx, ny, seed0 + b)
        h = min(1.0 / (nx + 1), 1.0 / (ny + 1))
        tau = 0.5 * h / math.sqrt(m.max())
        src = (nx // 2, ny // 3)
        wav = inputs.wavelet_samples(steps + 2, tau, fp=3.0)
        phi = smooth_state(nx, ny, 100 + b, 1e-2)
        out.append(dict(m=m, phi=phi, tau=tau, src=src, wav=wav, nx=nx, ny=ny))
    return out


def _run_batch(shots, steps, mode=0):
    import torch
    from paper_2006_10142_gb300 import api
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(f32(a)).to(dev)
    B = api.AdiWaveBatch([t(s["m"]) for s in shots], [t(s["phi"]) for s in shots],
                         [s["tau"] for s in shots])
    B.set_mode(mode)
    wavs = [t(s["wav"]) for s in shots]
    B.run(steps, srcs=[s["src"] for s in shots], wavelets=wavs)
    B.sync_status()
    res = [B.state(b) for b in range(len(shots))]
    out = [(up.double().cpu().numpy(), uc.double().cpu().numpy(), k) for up, uc, k in res]
    n_launch = B.launch_count()
    B.close()
    return out, n_launch


SHAPES = [(53, 37), (256, 256), (300, 128), (64, 64), (100, 200), (1000, 600), (17, 300)]


def test_batch_matches_oracle_per_shot():
    steps = 16
    shots = _shots(SHAPES, steps)
    got, _ = _run_batch(shots, steps)
    for b, s in enumerate(shots):
        o = oracle_run(s["m"], s["phi"], s["tau"], steps, src=s["src"], wavelet=s["wav"])
        assert got[b][2] == steps + 1
        e = rel_l2(got[b][1], o["u_cur"])
        assert e < 1e-4, (b, SHAPES[b], e)
        assert rel_l2(got[b][0], o["u_prev"]) < 1e-4


def test_parallel_branches_match_oracle_and_serial_launches():
    """Batch mode 2 (each shot's steps a chain on one of eight streams,
    replayed as parallel graph branches): per shot bit-exact with the serial
    per-shot launches of mode 1 (the same kernels) and within 1e-4 of the
    oracle; an odd step count exercises the graph pairs and a direct step."""
    steps = 9
    shots = _shots(SHAPES, steps, seed0=30)
    a, _ = _run_batch(shots, steps, mode=2)
    b, _ = _run_batch(shots, steps, mode=1)
    for s, sh in enumerate(shots):
        assert a[s][2] == steps + 1
        assert np.array_equal(a[s][1], b[s][1]) and np.array_equal(a[s][0], b[s][0]), s
        o = oracle_run(sh["m"], sh["phi"], sh["tau"], steps, src=sh["src"], wavelet=sh["wav"])
        assert rel_l2(a[s][1], o["u_cur"]) < 1e-4


def test_persistent_kernel_matches_per_shot_launches():
    steps = 9  # odd: four graph-replayed pairs and one direct step
    shots = _shots(SHAPES, steps, seed0=10)
    a, n_a = _run_batch(shots, steps, mode=0)
    b, n_b = _run_batch(shots, steps, mode=1)
    for s in range(len(shots)):
        assert rel_l2(a[s][1], b[s][1]) < 1e-5, s
    # one launch per step instead of two per shot and step
    assert n_a < n_b


def test_dependency_wait_times_out_without_fault():
    import torch
    from paper_2006_10142_gb300 import api
    shots = _shots(SHAPES[:3], 4, seed0=20)
    dev = torch.device("cuda:0")
    t = lambda a: torch.from_numpy(f32(a)).to(dev)
    B = api.AdiWaveBatch([t(s["m"]) for s in shots], [t(s["phi"]) for s in shots],
                         [s["tau"] for s in shots])
    B.set_mode(0)  # the persistent kernel's dependency wait
    B.set_wait_hook(spin_limit=2000, never_ready_shot=1)
    B.run(1)
    with pytest.raises(api.AdiError) as ei:
        B.sync_status()
    assert ei.value.code == 5  # ADI_ETIMEOUT
    # the context is still usable: clear the hook and step again
    B.set_wait_hook(0, -1)
    B.run(2)
    B.sync_status()
    up, uc, k = B.state(0)
    assert k == 4 and torch.isfinite(uc).all()
    B.close()


@pytest.mark.slow
def test_batch_64_shots_workload():
    """64 shots with n drawn from {256, 512, 1024, 2048}, 500 steps, in the
    default batch mode; three shots (256, 1024, 2048) checked against the
    oracle's full run."""
    import torch
    from paper_2006_10142_gb300 import api
    sizes = inputs.batch_sizes(64, seed=0)
    steps = 500
    dev = torch.device("cuda:0")
    probs = [inputs.ricker_problem(n, steps, seed=b, m_dtype=np.float32) for b, n in enumerate(sizes)]
    t = lambda a: torch.from_numpy(f32(a)).to(dev)
    B = api.AdiWaveBatch([t(p.m) for p in probs], [t(p.phi) for p in probs], [p.tau for p in probs])
    B.run(steps, srcs=[p.src for p in probs], wavelets=[t(p.wavelet) for p in probs])
    B.sync_status()
    picks = [sizes.index(256), sizes.index(1024), sizes.index(2048)]
    for b in picks:
        p = probs[b]
        _, uc, k = B.state(b)
        o = oracle_run(p.m, p.phi, p.tau, steps, src=p.src, wavelet=p.wavelet)
        assert k == steps + 1
        assert rel_l2(uc.double().cpu().numpy(), o["u_cur"]) < 1e-4, (b, sizes[b])
    B.close()
