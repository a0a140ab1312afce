"""The shot-parallel misfit gradient on one GPU (fwi.misfit_gradient with the
CUDA library per shot) against the FP64 oracle's sum over the same shots:
three shots share a seeded 64 x 64 medium, observed data from a perturbed
medium (oracle), relative L2 <= 1e-4 for dJ/dm and the misfit."""
import numpy as np
import pytest

import oracle
from paper_2006_10142_gb300 import fwi, inputs
from helpers import THREADS, f32, rel_l2

pytestmark = pytest.mark.gpu


def test_shot_gradients_sum_matches_oracle():
    import torch
    n, steps = 64, 150
    dev = torch.device("cuda:0")
    base, m_true = inputs.adjoint_problem(n, steps, seed=2, n_rec=16)
    m32 = f32(base.m)
    hx = 1.0 / (n + 1)
    z = np.zeros((n, n))
    wav = f32(base.wavelet)
    shots, ref_J, ref_g = [], 0.0, np.zeros((n, n))
    for s, x in enumerate((0.25, 0.5, 0.75)):
        src = (inputs.nearest_node(x, n), inputs.nearest_node(0.9, n))
        _, _, d = oracle.adi_run(f32(m_true).astype(np.float64), z, z, hx, hx, base.tau, steps,
                                 src=src, wavelet=wav.astype(np.float64), rec=base.rec,
                                 threads=THREADS)
        _, _, tr = oracle.adi_run(m32.astype(np.float64), z, z, hx, hx, base.tau, steps, src=src,
                                  wavelet=wav.astype(np.float64), rec=base.rec, threads=THREADS)
        resid = tr - d
        ref_J += 0.5 * float(np.sum(resid ** 2))
        ref_g += oracle.adi_adjoint(m32.astype(np.float64), z, z, hx, hx, base.tau, steps, resid,
                                    base.rec, src=src, wavelet=wav.astype(np.float64),
                                    threads=THREADS)["grad_m"]
        shots.append(fwi.Shot(src=src, wavelet=torch.from_numpy(wav).to(dev), rec=base.rec,
                              data=torch.from_numpy(f32(d)).to(dev)))
    J, g = fwi.misfit_gradient(torch.from_numpy(m32).to(dev), shots, base.tau, steps, every=50)
    assert ref_J > 0
    assert abs(J - ref_J) < 1e-4 * ref_J, (J, ref_J)
    assert rel_l2(g.cpu().numpy(), ref_g) < 1e-4
