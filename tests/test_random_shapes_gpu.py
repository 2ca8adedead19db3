"""Parity over seeded random stack shapes (ragged sizes, 1-3 lattices, padded
plane strides): the BGK step with totals and the GNN-LBM step against the
oracle, at the tolerances of the fixed-shape tests (BGK 1e-6 relative per
population after one step from identical FP32 input, totals 1e-12 of the
FP64 sum of the same values; GNN-LBM correction relative L2 <= 3e-2)."""
import numpy as np
import pytest

from oracle import gnn, lbm
from paper_2504_14494_gb300 import inputs
from gpu_util import from_dev, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _shapes(seed, count, max_nodes):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        nx, ny, nb = int(rng.integers(1, 300)), int(rng.integers(1, 40)), int(rng.integers(1, 4))
        if nx * ny * nb <= max_nodes:
            pad = int(rng.choice([0, 0, 4, 13]))
            out.append((nb, ny, nx, pad))
    return out


def _state(nb, ny, nx, seed):
    rng = np.random.default_rng(seed)
    f = np.stack([lbm.tgv_init(nx, ny, 1.0, 0.05, 2 * np.pi / nx, 2 * np.pi / ny)] * nb, axis=1)
    return (f * (1 + 2e-2 * rng.uniform(-1, 1, f.shape))).astype(np.float32)


@pytest.mark.parametrize("case", _shapes(11, 12, 40000))
def test_bgk_step_random_shapes(lbmlib, cuda, case):
    import torch
    L = lbmlib
    nb, ny, nx, pad = case
    n = nb * ny * nx
    f = _state(nb, ny, nx, seed=nx * 7 + ny)
    din, ps = to_dev(f, cuda, plane_stride=n + pad if pad else 0)
    dout = torch.zeros_like(din)
    tot = torch.zeros(5, dtype=torch.float64, device=cuda)
    s = L.shape(nx, ny, nb, ps)
    L.lbm_step_bgk(din, dout, None, s, 0.7, totals=tot)
    assert L.lbm_get_status() == 0
    got = from_dev(dout, f.shape, ps)
    ref = np.stack([lbm.bgk_step(f[:, b].astype(np.float64), 0.7) for b in range(nb)], axis=1)
    assert np.all(np.abs(got - ref) <= 1e-6 * np.abs(ref)), case
    t = tot.cpu().numpy()
    assert abs(t[0] - got.sum()) <= 1e-12 * got.sum(), case


@pytest.mark.parametrize("case", _shapes(12, 6, 5000))
def test_gnn_step_random_shapes(lbmlib, cuda, case):
    import torch
    L = lbmlib
    nb, ny, nx, pad = case
    n = nb * ny * nx
    f = _state(nb, ny, nx, seed=nx * 5 + ny)
    theta = inputs.xavier_params(nx + ny, s_df=1e-2, bias_scale=0.1)
    p = torch.from_numpy(theta).to(cuda)
    pk = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=cuda)
    L.gnn_pack(p, pk)
    din, ps = to_dev(f, cuda, plane_stride=n + pad if pad else 0)
    dout = torch.zeros_like(din)
    s = L.shape(nx, ny, nb, ps)
    ws = torch.empty(L.gnn_step_workspace_bytes(s), dtype=torch.uint8, device=cuda)
    L.lbm_step_gnn(din, dout, s, 0.7, None, pk, None, ws)
    assert L.lbm_get_status() == 0
    got = from_dev(dout, f.shape, ps)
    ref = np.stack([gnn.gnn_step(f[:, b].astype(np.float64), theta, 0.7) for b in range(nb)],
                   axis=1)
    bgk = np.stack([lbm.bgk_step(f[:, b].astype(np.float64), 0.7) for b in range(nb)], axis=1)
    assert rel_l2(got - bgk, ref - bgk) <= 3e-2, case
