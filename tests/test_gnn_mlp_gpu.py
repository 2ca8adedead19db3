"""The paper's Fig. 2 network (MLP-only variant) as one fused GNN-LBM step
kernel (lbm_step_gnn_mlp, and lbm_step_gnn on an MLP-only image), through
the C ABI, against the FP64 oracle's GNN step.

Tolerances (as the other GNN-LBM step tests: BF16 weights and activations,
FP32 accumulation and populations): relative L2 of the correction f* -
f*_BGK <= 3e-2, and per population |f* - f*_oracle| <= 1e-6 |f*_oracle| +
5e-2 max |f*_oracle - f*_BGK|.  lbm_step_gnn on an MLP-only image runs the
same kernel, so it must give the same bits.
"""
import numpy as np
import pytest

from oracle import gnn, lbm
from paper_2504_14494_gb300 import inputs
from gpu_util import from_dev, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _state(nb, ny, nx, seed, u0=0.05, amp=2e-2):
    f = np.stack([lbm.tgv_init(nx, ny, 1.0, u0, 2 * np.pi / nx, 2 * np.pi / ny)] * nb, axis=1)
    return (f * inputs.perturbation(f.shape, seed, amp)).astype(np.float32)


def _packed(L, theta, dev):
    import torch
    p = torch.from_numpy(np.asarray(theta, np.float32)).to(dev)
    pk = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=dev)
    L.gnn_pack(p, pk)
    return pk


def _check(got, f, theta, taus):
    nb = f.shape[1]
    ref = np.stack([gnn.gnn_step(f[:, b].astype(np.float64), theta, taus[b]) for b in range(nb)], 1)
    bgk = np.stack([lbm.bgk_step(f[:, b].astype(np.float64), taus[b]) for b in range(nb)], 1)
    e_corr = rel_l2(got - bgk, ref - bgk)
    e_f = np.max(np.abs(got - ref) - 1e-6 * np.abs(ref)) / np.max(np.abs(ref - bgk))
    print(f"correction rel L2 {e_corr:.2e}; max err / max correction {e_f:.2e}")
    assert e_corr <= 3e-2 and e_f <= 5e-2, (e_corr, e_f)


# ragged last tiles, 1x1, wraps in x and y, stacks, a padded plane stride
@pytest.mark.parametrize("nb,ny,nx,pad,variant", [
    (1, 16, 16, 0, 1), (1, 1, 1, 0, 1), (2, 5, 7, 0, 3), (1, 12, 130, 0, 1), (3, 9, 64, 37, 3),
    (1, 33, 128, 0, 5), (2, 20, 24, 0, 7), (2, 4, 256, 0, 3), (1, 3, 384, 4, 1),
    (1, 1, 128, 0, 3)])
def test_fused_mlp_step_matches_oracle(lbmlib, cuda, nb, ny, nx, pad, variant):
    import torch
    L = lbmlib
    theta = inputs.xavier_params(90 + nx, s_df=1e-2, bias_scale=0.1, variant=variant)
    f = _state(nb, ny, nx, seed=nx + 5 * ny)
    n = nb * ny * nx
    din, ps = to_dev(f, cuda, plane_stride=(n + pad) if pad else 0)
    s = L.shape(nx, ny, nb, ps if pad else 0)
    taus = [0.55 + 0.2 * b for b in range(nb)]
    td = torch.tensor(taus, dtype=torch.float32, device=cuda)
    pk = _packed(L, theta, cuda)
    out = torch.full_like(din, float("nan"))
    tot = torch.zeros(5, dtype=torch.float64, device=cuda)
    L.lbm_step_gnn_mlp(din, out, s, 1.0, td, pk, tot)
    assert L.lbm_get_status() == 0
    got = from_dev(out, f.shape, ps)
    assert np.isfinite(got).all()
    _check(got, f, theta, taus)
    # lbm_step_gnn takes the same kernel for an MLP-only image
    ws = torch.empty(L.gnn_step_workspace_bytes(s), dtype=torch.uint8, device=cuda)
    out2 = torch.full_like(din, float("nan"))
    L.lbm_step_gnn(din, out2, s, 1.0, td, pk, None, ws)
    assert L.lbm_get_status() == 0
    assert torch.equal(out.view(9, ps)[:, :n], out2.view(9, ps)[:, :n])
    t_ref = sum(lbm.totals(got[:, b]) for b in range(nb))
    assert abs(tot[0].item() - t_ref[0]) <= 1e-12 * t_ref[0]


@pytest.mark.parametrize("nb,ny,nx", [(2, 6, 256), (1, 1, 128), (1, 5, 512), (3, 2, 128)])
def test_fused_mlp_row_runs_equal_node_pulls(lbmlib, cuda, nb, ny, nx):
    """Rows of whole tiles with 16-byte aligned planes take the row-run fetch
    (each population's source run of a tile in 16-byte chunks); a plane
    stride that is not a multiple of 4 takes the per-node 4-byte pulls.  The
    arithmetic after the fetch is the same, so the two give the same bits."""
    import torch
    L = lbmlib
    theta = inputs.xavier_params(95 + ny, s_df=1e-2, bias_scale=0.1, variant=3)
    f = _state(nb, ny, nx, seed=nx + ny)
    n = nb * ny * nx
    pk = _packed(L, theta, cuda)
    td = torch.tensor([0.6 + 0.1 * b for b in range(nb)], dtype=torch.float32, device=cuda)
    outs = []
    for ps in (n, n + 1):
        din, _ = to_dev(f, cuda, plane_stride=ps)
        out = torch.full_like(din, float("nan"))
        L.lbm_step_gnn_mlp(din, out, L.shape(nx, ny, nb, ps), 1.0, td, pk, None)
        assert L.lbm_get_status() == 0
        outs.append(out.view(9, ps)[:, :n])
    assert torch.equal(outs[0], outs[1])
    _check(from_dev(outs[0].reshape(-1), f.shape), f, theta, [0.6 + 0.1 * b for b in range(nb)])


def test_fused_mlp_step_refuses_a_message_passing_image(lbmlib, cuda):
    import torch
    L = lbmlib
    f = _state(1, 8, 12, seed=3)
    din, _ = to_dev(f, cuda)
    out = torch.full_like(din, -5.0)
    pk = _packed(L, inputs.xavier_params(4, variant=0), cuda)
    L.lbm_step_gnn_mlp(din, out, L.shape(12, 8), 0.7, None, pk, None)
    assert L.lbm_get_status() == L.LBM_ERR_BLOB
    assert bool((out == -5.0).all())


def test_fused_mlp_step_full_size_4096_sampled(lbmlib, cuda):
    """The 4096^2 lattice the benchmark times for this network: 200 sampled
    nodes, the corners and edge nodes against the oracle's step of the 3 x 3
    periodic patch around each (the MLP-only network is local: the result at
    a node depends on the populations pulled into it only)."""
    import torch
    L = lbmlib
    n = 4096
    s = L.shape(n, n)
    k = 2 * np.pi / n
    theta = inputs.xavier_params(5, s_df=1e-2, bias_scale=0.1, variant=3)
    pk = _packed(L, theta, cuda)
    f = torch.empty(9 * n * n, device=cuda)
    L.lbm_init_tgv(f, s, 1.0, 0.05, k, k, False)
    g = torch.Generator(device=cuda)
    g.manual_seed(7)
    f.mul_(1.0 + 2e-2 * (2.0 * torch.rand(f.shape, generator=g, device=cuda) - 1.0))
    out = torch.empty_like(f)
    L.lbm_step_gnn_mlp(f, out, s, 0.6, None, pk, None)
    assert L.lbm_get_status() == 0
    rng = np.random.default_rng(11)
    pts = [(0, 0), (0, n - 1), (n - 1, 0), (n - 1, n - 1), (n // 2, 0), (0, n // 2)]
    pts += [tuple(int(v) for v in rng.integers(0, n, 2)) for _ in range(200)]
    F = f.view(9, n, n)
    O = out.view(9, n, n)
    got, ref, bgk = [], [], []
    for (y, x) in pts:
        ys = [(y + d) % n for d in (-1, 0, 1)]
        xs = [(x + d) % n for d in (-1, 0, 1)]
        patch = F[:, ys][:, :, xs].cpu().numpy().astype(np.float64)
        ref.append(gnn.gnn_step(patch, theta, 0.6)[:, 1, 1])
        bgk.append(lbm.bgk_step(patch, 0.6)[:, 1, 1])
        got.append(O[:, y, x].cpu().numpy().astype(np.float64))
    got, ref, bgk = np.array(got), np.array(ref), np.array(bgk)
    e_corr = rel_l2(got - bgk, ref - bgk)
    e_f = np.max(np.abs(got - ref) - 1e-6 * np.abs(ref)) / np.max(np.abs(ref - bgk))
    assert e_corr <= 3e-2 and e_f <= 5e-2, (e_corr, e_f)


def test_batched_run_of_mlp_only_network(lbmlib, cuda):
    """Batched uneven lattices with the Fig. 2 network (the fused kernel over
    the lattice table): every lattice equals its own lbm_step_gnn_mlp run."""
    import torch
    L = lbmlib
    lat = [(8, 8, 1, 0.8), (13, 7, 1, 0.7), (32, 32, 0, 0.55), (130, 3, 1, 0.9), (1, 1, 1, 0.75)]
    theta = inputs.xavier_params(23, s_df=1e-2, bias_scale=0.1, variant=1)
    pk = _packed(L, theta, cuda)
    plan = L.lbm_batch_plan_create(lat)
    try:
        n = L.lbm_batch_nodes(plan)
        off = L.lbm_batch_offsets(plan, len(lat))
        prm = np.array([(1.0, 0.03, 2 * np.pi / nx, 2 * np.pi / ny) for nx, ny, _, _ in lat])
        f0 = torch.empty(9 * n, device=cuda)
        L.lbm_batch_init_tgv(plan, f0, prm, False)
        f1, f2 = torch.empty_like(f0), torch.empty_like(f0)
        ws = torch.empty(max(L.lbm_batch_workspace_bytes(plan), 16), dtype=torch.uint8,
                         device=cuda)
        L.lbm_batch_run(plan, f0, f1, f2, 2, pk, ws)
        assert L.lbm_get_status() == 0
        F0, F1 = f0.view(9, n), f1.view(9, n)
        for i, (nx, ny, col, tau) in enumerate(lat):
            m = nx * ny
            a = F0[:, off[i]:off[i] + m].contiguous().reshape(-1)
            b = torch.empty_like(a)
            s = L.shape(nx, ny)
            for _ in range(2):
                if col == 0:
                    L.lbm_step_bgk(a, b, None, s, tau)
                else:
                    L.lbm_step_gnn_mlp(a, b, s, tau, None, pk, None)
                a, b = b, a
            assert torch.allclose(F1[:, off[i]:off[i] + m].reshape(-1), a, rtol=1e-6, atol=0), i
    finally:
        L.lbm_batch_plan_destroy(plan)
