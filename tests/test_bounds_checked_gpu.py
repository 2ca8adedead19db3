"""The bounds-checked test build (liblbmgnn_checked.so, -DLBM_BOUNDS_CHECK:
every computed gather index is checked against its buffer and a failed check
raises the status word's bounds bit instead of reading out of range) runs the
kernels on small and degenerate shapes without a single failed check, and
gives bitwise the results of the regular build."""
import numpy as np
import pytest

from oracle import lbm
from paper_2504_14494_gb300 import inputs
from gpu_util import to_dev

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (1, 3, 5), (2, 5, 7), (1, 16, 24), (1, 6, 128), (3, 4, 130), (2, 8, 16),
          (2, 3, 256)]


def _state(nb, ny, nx, seed):
    f = np.stack([lbm.tgv_init(nx, ny, 1.0, 0.05, 2 * np.pi / nx, 2 * np.pi / ny)] * nb, axis=1)
    return (f * inputs.perturbation(f.shape, seed, 2e-2)).astype(np.float32)


def _scenario(L, dev):
    """Runs every kernel family on SHAPES; returns the outputs and the status."""
    import torch
    out = []
    theta = inputs.xavier_params(7, s_df=1e-2, bias_scale=0.1)
    p = torch.from_numpy(theta).to(dev)
    pk = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=dev)
    L.gnn_pack(p, pk)
    # the paper's Fig. 2 network for the fused step (row-run fetch where the
    # rows are whole tiles, per-node pulls elsewhere)
    pk_mlp = torch.empty_like(pk)
    L.gnn_pack(torch.from_numpy(inputs.xavier_params(8, s_df=1e-2, bias_scale=0.1,
                                                     variant=3)).to(dev), pk_mlp)
    for (nb, ny, nx) in SHAPES:
        f = _state(nb, ny, nx, seed=nx + ny)
        din, _ = to_dev(f, dev)
        s = L.shape(nx, ny, nb)
        a, b = torch.empty_like(din), torch.empty_like(din)
        tot = torch.zeros(5, dtype=torch.float64, device=dev)
        L.lbm_step_bgk(din, a, b, s, 0.7, nsteps=3, totals=tot)
        out += [a.clone(), tot.clone()]
        L.lbm_step_channel(din, a, b, s, 0.8, None, 1e-5, 2)
        out.append(a.clone())
        ws = torch.empty(L.gnn_step_workspace_bytes(s), dtype=torch.uint8, device=dev)
        L.lbm_step_gnn(din, a, s, 0.75, None, pk, None, ws)
        out.append(a.clone())
        L.lbm_step_gnn_mlp(din, a, s, 0.75, None, pk_mlp, None)
        out.append(a.clone())
        wc = torch.empty(L.gnn_channel_workspace_bytes(s), dtype=torch.uint8, device=dev)
        L.lbm_step_gnn_channel(din, a, s, 0.8, None, 1e-5, pk, None, wc)
        out.append(a.clone())
        # training path: forward, Eq. 3 + Eq. 4, backward (edge-term gathers)
        n = nb * ny * nx
        saved = torch.empty(L.gnn_saved_bytes(s), dtype=torch.uint8, device=dev)
        y = torch.empty(10 * n, device=dev)
        dy = torch.empty(10 * n, device=dev)
        loss = torch.zeros(1, dtype=torch.float64, device=dev)
        L.gnn_forward(din, s, pk, saved, y)
        wl = torch.empty(L.gnn_loss_workspace_bytes(s), dtype=torch.uint8, device=dev)
        L.gnn_collide_loss(din, y, a, s, 0.75, None, pk, loss, dy, None, wl)
        g = torch.empty(L.gnn_trainable_count(), device=dev)
        wb = torch.empty(L.gnn_backward_workspace_bytes(s), dtype=torch.uint8, device=dev)
        L.gnn_backward(din, s, pk, saved, dy, g, None, wb)
        out += [y.clone(), g.clone()]
        # channel training: forced restriction of a 3x refined channel, and
        # the fused step (walled edge backward, forced encoder backward)
        ff, _ = to_dev(_state(nb, 3 * ny, 3 * nx, seed=nx + 2 * ny), dev)
        L.lbm_restrict_channel(ff, L.shape(3 * nx, 3 * ny, nb), b, s, 3, 0.9, None, 0.6333333,
                               None, 2e-5)
        out.append(b.clone())
        pc, pkc = p.clone(), pk.clone()
        mc, vc = torch.zeros_like(g), torch.zeros_like(g)
        wt = torch.empty(L.gnn_train_workspace_bytes(s), dtype=torch.uint8, device=dev)
        L.gnn_train_step_channel(din, b, s, 0.75, None, 6e-5, None, None, pc, pkc, mc, vc, 1, 1e-3,
                                 1e-2, loss, g, wt)
        out += [loss.clone(), g.clone(), pc.clone()]
    # batched run (table geometry)
    lat = [(5, 3, 0, 0.7), (130, 2, 1, 0.8), (1, 1, 1, 0.9), (24, 16, 1, 0.65)]
    plan = L.lbm_batch_plan_create(lat)
    try:
        n = L.lbm_batch_nodes(plan)
        prm = np.array([(1.0, 0.03, 2 * np.pi / l[0], 2 * np.pi / l[1]) for l in lat])
        f0 = torch.empty(9 * n, device=dev)
        L.lbm_batch_init_tgv(plan, f0, prm, False)
        f1, f2 = torch.empty_like(f0), torch.empty_like(f0)
        ws = torch.empty(max(L.lbm_batch_workspace_bytes(plan), 16), dtype=torch.uint8, device=dev)
        L.lbm_batch_run(plan, f0, f1, f2, 2, pk, ws)
        out.append(f1.clone())
    finally:
        L.lbm_batch_plan_destroy(plan)
    return out, L.lbm_get_status()


def test_checked_build_finds_no_bad_index_and_matches(lbmlib, cuda):
    import torch
    from paper_2504_14494_gb300 import build, lib as L
    path = build.build(checked=True)
    regular = L._lib
    L._lib = None
    try:  # the checked build first: a bad index is then reported, not read
        L.load(path)
        got, st = _scenario(L, cuda)
        assert st == 0, L.status_string(st)   # LBM_ERR_BOUNDS: a gather index out of range
    finally:
        L._lib = regular
    want, st = _scenario(L, cuda)
    assert st == 0
    assert len(got) == len(want)
    for i, (a, b) in enumerate(zip(got, want)):
        assert torch.equal(a, b), i
