"""The packed parameter image's validity word (gnn_pack; include/lbmgnn.h):
an image that was never packed, or was packed from invalid fixed values
(variant outside 0..7, sigma or s_df not > 0, a non-finite normaliser), is
refused by every kernel that reads it: nothing is written, a loss becomes
NaN, and lbm_get_status() reports LBM_ERR_BLOB.  A valid pack afterwards
works as before.  (Error path of the boundary: the paper's method has no
counterpart.)"""
import numpy as np
import pytest

from oracle import lbm
from paper_2504_14494_gb300 import inputs

pytestmark = pytest.mark.gpu

NX, NY, NB = 16, 8, 2


def _dev_state(torch, cuda):
    f = lbm.tgv_init(NX, NY, 1.0, 0.05, 2 * np.pi / NX, 2 * np.pi / NY)
    f = np.stack([f] * NB, axis=1).astype(np.float32)
    return torch.from_numpy(f.reshape(-1).copy()).to(cuda)


def _pack(L, torch, cuda, theta):
    p = torch.from_numpy(np.asarray(theta, np.float32)).to(cuda)
    pk = torch.zeros(L.gnn_packed_bytes(), dtype=torch.uint8, device=cuda)
    L.gnn_pack(p, pk)
    return p, pk


def test_unpacked_image_is_refused_by_every_kernel(lbmlib, cuda):
    import torch
    L = lbmlib
    assert L.lbm_get_status() == L.LBM_OK
    s = L.shape(NX, NY, NB)
    n = NX * NY * NB
    f = _dev_state(torch, cuda)
    zero = torch.zeros(L.gnn_packed_bytes(), dtype=torch.uint8, device=cuda)
    # inference step (and its internal-scratch twin)
    out = torch.full_like(f, -7.0)
    ws = torch.empty(L.gnn_step_workspace_bytes(s), dtype=torch.uint8, device=cuda)
    L.lbm_step_gnn(f, out, s, 0.8, None, zero, None, ws)
    assert L.lbm_get_status() == L.LBM_ERR_BLOB
    assert bool((out == -7.0).all())
    L.lbm_step_gnn_noalloc(f, out, s, 0.8, None, zero, None)
    assert L.lbm_get_status() == L.LBM_ERR_BLOB
    assert bool((out == -7.0).all())
    # channel step (walls, Guo forcing)
    wc = torch.empty(L.gnn_channel_workspace_bytes(s), dtype=torch.uint8, device=cuda)
    L.lbm_step_gnn_channel(f, out, s, 0.8, None, 1e-3, zero, None, wc)
    assert L.lbm_get_status() == L.LBM_ERR_BLOB
    assert bool((out == -7.0).all())
    # training forward, Eq. 3 + Eq. 4, backward, fused step
    saved = torch.empty(L.gnn_saved_bytes(s), dtype=torch.uint8, device=cuda)
    y = torch.full((10 * n,), -7.0, device=cuda)
    L.gnn_forward(f, s, zero, saved, y)
    assert L.lbm_get_status() == L.LBM_ERR_BLOB
    assert bool((y == -7.0).all())
    loss = torch.zeros(1, dtype=torch.float64, device=cuda)
    dy = torch.zeros(10 * n, device=cuda)
    wl = torch.empty(L.gnn_loss_workspace_bytes(s), dtype=torch.uint8, device=cuda)
    L.gnn_collide_loss(f, torch.zeros(10 * n, device=cuda), f, s, 0.8, None, zero, loss, dy,
                       None, wl)
    assert L.lbm_get_status() == L.LBM_ERR_BLOB
    assert bool(torch.isnan(loss).all())
    grad = torch.zeros(L.gnn_trainable_count(), device=cuda)
    wb = torch.empty(L.gnn_backward_workspace_bytes(s), dtype=torch.uint8, device=cuda)
    L.gnn_backward(f, s, zero, saved, dy, grad, None, wb)
    assert L.lbm_get_status() == L.LBM_ERR_BLOB
    theta = inputs.xavier_params(3, s_df=1e-3)
    p = torch.from_numpy(theta).to(cuda)
    m = torch.zeros(L.gnn_trainable_count(), device=cuda)
    v = torch.zeros_like(m)
    wt = torch.empty(L.gnn_train_workspace_bytes(s), dtype=torch.uint8, device=cuda)
    L.gnn_train_step(f, f, s, 0.8, None, p, zero, m, v, 1, 1e-3, 0.0, loss, None, wt)
    assert L.lbm_get_status() == L.LBM_ERR_BLOB
    assert bool(torch.isnan(loss).all())
    # the fused step re-packs the (unchanged, valid) parameters at its end
    L.lbm_step_gnn(f, out, s, 0.8, None, zero, None, ws)
    assert L.lbm_get_status() == L.LBM_OK
    assert bool(torch.isfinite(out).all())
    # batched run
    plan = L.lbm_batch_plan_create([(NX, NY, 1, 0.8), (8, 8, 0, 0.7)])
    try:
        nb_ = L.lbm_batch_nodes(plan)
        fb = torch.ones(9 * nb_, device=cuda) / 9
        ob = torch.full_like(fb, -7.0)
        wsb = torch.empty(L.lbm_batch_workspace_bytes(plan), dtype=torch.uint8, device=cuda)
        L.lbm_batch_run(plan, fb, ob, None, 1, zero, wsb)  # valid image: the autotuner runs here
        assert L.lbm_get_status() == L.LBM_OK
        ob.fill_(-7.0)
        bad = torch.zeros_like(zero)
        L.lbm_batch_run(plan, fb, ob, None, 1, bad, wsb)
        assert L.lbm_get_status() == L.LBM_ERR_BLOB
        off = L.lbm_batch_offsets(plan, 2)
        assert bool((ob.view(9, nb_)[:, off[0]:off[0] + NX * NY] == -7.0).all())  # GNN lattice
        assert bool((ob.view(9, nb_)[:, off[1]:off[1] + 64] != -7.0).all())      # BGK lattice
    finally:
        L.lbm_batch_plan_destroy(plan)


@pytest.mark.parametrize("what", ["variant", "sigma", "s_df", "mu"])
def test_invalid_fixed_values_are_refused(lbmlib, cuda, what):
    import torch
    L = lbmlib
    s = L.shape(NX, NY, NB)
    f = _dev_state(torch, cuda)
    theta = inputs.xavier_params(4, s_df=1e-2)
    o = inputs.N_TRAINABLE  # mu[12], sigma[12], s_df, variant
    bad = theta.copy()
    if what == "variant":
        bad[o + 25] = 8.0
    elif what == "sigma":
        bad[o + 12 + 3] = 0.0
    elif what == "s_df":
        bad[o + 24] = -1e-2
    else:
        bad[o + 5] = np.nan
    _, pk = _pack(L, torch, cuda, bad)
    assert L.lbm_get_status() == L.LBM_ERR_BLOB
    out = torch.full_like(f, -7.0)
    ws = torch.empty(L.gnn_step_workspace_bytes(s), dtype=torch.uint8, device=cuda)
    L.lbm_step_gnn(f, out, s, 0.8, None, pk, None, ws)
    assert L.lbm_get_status() == L.LBM_ERR_BLOB
    assert bool((out == -7.0).all())
    # the valid vector packs and steps
    _, pk = _pack(L, torch, cuda, theta)
    L.lbm_step_gnn(f, out, s, 0.8, None, pk, None, ws)
    assert L.lbm_get_status() == L.LBM_OK
    assert bool(torch.isfinite(out).all())
