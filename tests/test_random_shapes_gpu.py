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


@pytest.mark.parametrize("case", _shapes(13, 4, 1500))
def test_gnn_backward_random_shapes(lbmlib, cuda, case):
    """gnn_backward against the oracle's FP64 backward: per parameter tensor
    cosine >= 0.999 and relative L2 <= 3e-2, dL/df_pre the same."""
    import torch
    L = lbmlib
    nb, ny, nx, pad = case
    n = nb * ny * nx
    f = _state(nb, ny, nx, seed=nx * 3 + ny)
    theta = inputs.xavier_params(nx + 2 * ny, s_df=1e-2, bias_scale=0.1)
    p = torch.from_numpy(theta).to(cuda)
    pk = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=cuda)
    L.gnn_pack(p, pk)
    din, ps = to_dev(f, cuda, plane_stride=n + pad if pad else 0)
    s = L.shape(nx, ny, nb, ps)
    saved = torch.empty(L.gnn_saved_bytes(s), dtype=torch.uint8, device=cuda)
    y = torch.empty(10 * n, device=cuda)
    L.gnn_forward(din, s, pk, saved, y)
    dy = np.random.default_rng(n).standard_normal((n, 10))
    dyd = torch.from_numpy(dy.T.astype(np.float32).copy()).to(cuda).reshape(-1)
    grad = torch.zeros(L.gnn_trainable_count(), device=cuda)
    df = torch.zeros_like(din)
    ws = torch.empty(L.gnn_backward_workspace_bytes(s), dtype=torch.uint8, device=cuda)
    L.gnn_backward(din, s, pk, saved, dyd, grad, df, ws)
    assert L.lbm_get_status() == 0
    pr = gnn.unpack(theta)
    g_ref = np.zeros(gnn.N_TRAINABLE)
    df_ref = np.zeros(f.shape)
    per = ny * nx
    for b in range(nb):
        _, cache = gnn.forward(f[:, b].astype(np.float64), pr)
        gb, dfb = gnn.backward(dy[b * per:(b + 1) * per], cache, pr)
        g_ref += gnn.pack_grads(gb)
        df_ref[:, b] = dfb.reshape(9, ny, nx)
    g_gpu = grad.cpu().numpy().astype(np.float64)
    o = 0
    for name, shape in gnn.SHAPES:
        k = int(np.prod(shape))
        a, r = g_gpu[o:o + k], g_ref[o:o + k]
        o += k
        c = float(np.dot(a, r) / (np.linalg.norm(a) * np.linalg.norm(r) + 1e-300))
        assert c >= 0.999 and rel_l2(a, r) <= 3e-2, (case, name, c, rel_l2(a, r))
    assert rel_l2(from_dev(df, f.shape, ps), df_ref) <= 3e-2


@pytest.mark.parametrize("seed", [21, 22])
def test_random_batch_plans_equal_single_runs(lbmlib, cuda, seed):
    """A plan of 40 random lattices (sides 1-40, either collision, random
    tau): every lattice of two batched steps equals two single-lattice
    steps to FP32 rounding (1e-6)."""
    import torch
    L = lbmlib
    rng = np.random.default_rng(seed)
    lat = [(int(rng.integers(1, 41)), int(rng.integers(1, 41)), int(rng.integers(0, 2)),
            float(rng.uniform(0.55, 1.2))) for _ in range(40)]
    theta = inputs.xavier_params(seed, s_df=1e-2, bias_scale=0.1)
    p = torch.from_numpy(theta).to(cuda)
    pk = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=cuda)
    L.gnn_pack(p, pk)
    plan = L.lbm_batch_plan_create(lat)
    try:
        n = L.lbm_batch_nodes(plan)
        off = L.lbm_batch_offsets(plan, len(lat))
        prm = np.array([(1.0, 0.04, 2 * np.pi / l[0], 2 * np.pi / l[1]) for l in lat])
        f0 = torch.empty(9 * n, device=cuda)
        L.lbm_batch_init_tgv(plan, f0, prm, False)
        f1, f2 = torch.empty_like(f0), torch.empty_like(f0)
        ws = torch.empty(max(L.lbm_batch_workspace_bytes(plan), 16), dtype=torch.uint8,
                         device=cuda)
        L.lbm_batch_run(plan, f0, f1, f2, 2, pk, ws)
        assert L.lbm_get_status() == 0
        for i, (nx, ny, col, tau) in enumerate(lat):
            m = nx * ny
            a = f0.view(9, n)[:, off[i]:off[i] + m].contiguous().reshape(-1)
            b = torch.empty_like(a)
            s = L.shape(nx, ny)
            w = torch.empty(max(L.gnn_step_workspace_bytes(s), 16), dtype=torch.uint8,
                            device=cuda)
            for _ in range(2):
                if col == 0:
                    L.lbm_step_bgk(a, b, None, s, tau)
                else:
                    L.lbm_step_gnn(a, b, s, tau, None, pk, None, w)
                a, b = b, a
            got = f1.view(9, n)[:, off[i]:off[i] + m]
            assert torch.allclose(got, a.view(9, m), rtol=1e-6, atol=0), (i, nx, ny, col)
    finally:
        L.lbm_batch_plan_destroy(plan)
