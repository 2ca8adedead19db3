"""Parity of the CUDA channel (Poiseuille) step with the FP64 oracle:
one step from an identical FP32 input per population <= 1e-6 relative; the
profile after 3,000 steps within 2e-4 of the oracle's, relative to the
centre-line velocity: the FP32 iteration settles on a fixed point shifted by
about ulp(f) / (1 - lambda), ulp(0.44) = 3e-8 and 1 - lambda = nu pi^2 / H^2
= 0.026 for the slowest diffusive mode, i.e. ~1.2e-6 absolute, 2.4e-5 of the
4.8e-2 centre-line velocity (bound with a factor 8 of margin); mass
conservation to FP32 rounding."""
import numpy as np
import pytest

from oracle import channel, lbm
from paper_2504_14494_gb300 import inputs
from gpu_util import from_dev, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nb,ny,nx", [(1, 6, 4), (2, 7, 5), (1, 1, 3), (1, 32, 130)])
def test_channel_step_matches_oracle(lbmlib, cuda, nb, ny, nx):
    import torch
    L = lbmlib
    f = np.stack([lbm.equilibrium(np.ones((ny, nx)), np.full((ny, nx), 0.02), np.zeros((ny, nx)))] * nb, axis=1)
    f = (f * inputs.perturbation(f.shape, nx + ny, 1e-2)).astype(np.float32)
    taus = np.array([0.7, 1.1][:nb], np.float32)
    din, _ = to_dev(f, cuda)
    dout = torch.zeros_like(din)
    L.lbm_step_channel(din, dout, None, L.shape(nx, ny, nb), 0.0, torch.from_numpy(taus).to(cuda), 1e-4)
    got = from_dev(dout, f.shape)
    for b in range(nb):
        ref = channel.channel_step(f[:, b].astype(np.float64), float(taus[b]), 1e-4)
        assert np.all(np.abs(got[:, b] - ref) <= 1e-6 * np.abs(ref)), b


def test_channel_steady_profile_matches_oracle(lbmlib, cuda):
    import torch
    L = lbmlib
    ny, nx, tau, g = 8, 2, 1.0, 1e-3
    f0 = lbm.equilibrium(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx))).astype(np.float32)
    din, _ = to_dev(f0, cuda)
    a, b = torch.zeros_like(din), torch.zeros_like(din)
    tot = torch.zeros(5, dtype=torch.float64, device=cuda)
    L.lbm_step_channel(din, a, b, L.shape(nx, ny), tau, None, g, 3000, tot)
    assert L.lbm_get_status() == 0
    got = from_dev(a, f0.shape)
    ref = channel.channel_run(f0.astype(np.float64), tau, g, 3000)
    _, ug, _ = channel.moments_forced(got, g)
    _, ur, _ = channel.moments_forced(ref, g)
    assert np.abs(ug - ur).max() <= 2e-4 * np.abs(ur).max()
    assert abs(tot[0].item() - ny * nx) <= 1e-5 * ny * nx
