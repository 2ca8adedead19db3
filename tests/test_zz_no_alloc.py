"""lbm_step_gnn_noalloc: the GNN-LBM step for callers that cannot allocate
device memory (an application whose allocator owns the device, a loop that
may not allocate once running, a binding without device buffers).  It takes
its scratch from a fixed array inside the library instead of a workspace
argument.

Checked through the C ABI against lbm_step_gnn with a caller-provided
workspace on consecutive calls: the largest stack the array holds first, then
smaller ones, so the later calls run on the array with the earlier call's
contents left in it.  The same kernels on the same inputs must give the same
bits (torch.equal), including with a padded plane stride and per-lattice
relaxation times; one case is also checked against the FP64 oracle's GNN
step at the tolerances of the other GNN-LBM step tests.  The size limit is
enforced before any launch.

This file is collected last on purpose, so that a run stopping at the first
failure has run every other test first; it also passes alone.
"""
import numpy as np
import pytest

from oracle import gnn, lbm
from paper_2504_14494_gb300 import inputs
from gpu_util import from_dev, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _state(nb, ny, nx, seed):
    f = np.stack([lbm.tgv_init(nx, ny, 1.0, 0.05, 2 * np.pi / nx, 2 * np.pi / ny)] * nb, axis=1)
    return (f * inputs.perturbation(f.shape, seed, 2e-2)).astype(np.float32)


def test_noalloc_step_equals_workspace_step_on_consecutive_calls(lbmlib, cuda):
    import torch
    L = lbmlib
    theta = inputs.xavier_params(77, s_df=1e-3, bias_scale=0.1)
    params = torch.from_numpy(theta).to(cuda)
    packed = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=cuda)
    L.gnn_pack(params, packed)
    # (nb, ny, nx, tau or per-lattice taus, plane-stride padding); the first
    # case fills the array to its limit, the later ones reuse it
    cases = [(2, 128, 128, 0.65, 0),
             (1, 80, 96, 0.8, 0),
             (3, 40, 52, [0.6, 0.9, 0.7], 1000)]
    assert 2 * 128 * 128 == L.LBM_STEP_GNN_NOALLOC_MAX_NODES
    for (nb, ny, nx, tau, pad) in cases:
        f = _state(nb, ny, nx, seed=nx + ny)
        n = nb * ny * nx
        fin, ps = to_dev(f, cuda, plane_stride=(n + pad) if pad else 0)
        s = L.shape(nx, ny, nb, ps if pad else 0)
        taus = None
        tau0 = tau
        if isinstance(tau, list):
            taus = torch.tensor(tau, dtype=torch.float32, device=cuda)
            tau0 = 1.0
        ref = torch.full_like(fin, float("nan"))
        ws = torch.empty(L.gnn_step_workspace_bytes(s), dtype=torch.uint8, device=cuda)
        tot_ref = torch.zeros(5, dtype=torch.float64, device=cuda)
        L.lbm_step_gnn(fin, ref, s, tau0, taus, packed, tot_ref, ws)
        got = torch.full_like(fin, float("nan"))
        tot = torch.zeros(5, dtype=torch.float64, device=cuda)
        L.lbm_step_gnn_noalloc(fin, got, s, tau0, taus, packed, tot)
        assert L.lbm_get_status() == 0
        # padding between the planes is left as the caller wrote it (NaN)
        g = got.view(9, ps)[:, :n]
        assert torch.isfinite(g).all()
        assert torch.equal(g, ref.view(9, ps)[:, :n]), (nb, ny, nx)
        assert torch.equal(tot, tot_ref)
        if (nb, ny, nx) == (1, 80, 96):  # the oracle's GNN step on the same inputs
            got_np = from_dev(got, f.shape)
            ref_o = gnn.gnn_step(f[:, 0].astype(np.float64), theta, tau)
            bgk = lbm.bgk_step(f[:, 0].astype(np.float64), tau)
            e_corr = rel_l2(got_np[:, 0] - bgk, ref_o - bgk)
            corr = np.max(np.abs(ref_o - bgk))
            e_f = np.max(np.abs(got_np[:, 0] - ref_o) - 1e-6 * np.abs(ref_o)) / corr
            assert e_corr <= 3e-2, e_corr
            assert e_f <= 5e-2, e_f


def test_noalloc_rejects_oversize(lbmlib, cuda):
    import torch
    L = lbmlib
    n = L.LBM_STEP_GNN_NOALLOC_MAX_NODES + 1
    f = torch.zeros(9 * n, device=cuda)
    g = torch.zeros(9 * n, device=cuda)
    packed = torch.zeros(L.gnn_packed_bytes(), dtype=torch.uint8, device=cuda)
    with pytest.raises(L.LbmError) as e:
        L.lbm_step_gnn_noalloc(f, g, L.shape(n, 1, 1), 0.8, None, packed, None)
    assert e.value.code == -3
