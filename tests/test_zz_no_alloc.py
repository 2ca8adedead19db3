"""lbm_step_gnn_noalloc: the GNN-LBM step for callers that cannot allocate
device memory (an application whose allocator owns the device, a loop that
may not allocate once running, a binding without device buffers).  It takes
its scratch from a fixed array inside the library instead of a workspace
argument.

Checked through the C ABI against lbm_step_gnn (caller-provided workspace)
on two calls in a row -- the second on another shape, up to the size limit,
since the shared array keeps the first call's contents -- within the
tolerance the GNN step tests use for identical arithmetic (1e-6 relative per
population), and the size limit is enforced before any launch.

This file is collected last on purpose, so that a run stopping at the first
failure has run every other test first; it also passes alone.
"""
import numpy as np
import pytest

from oracle import lbm
from paper_2504_14494_gb300 import inputs
from gpu_util import to_dev

pytestmark = pytest.mark.gpu


def _state(nb, ny, nx, seed):
    f = np.stack([lbm.tgv_init(nx, ny, 1.0, 0.05, 2 * np.pi / nx, 2 * np.pi / ny)] * nb, axis=1)
    return (f * inputs.perturbation(f.shape, seed, 2e-2)).astype(np.float32)


def test_noalloc_step_matches_workspace_step_twice(lbmlib, cuda):
    import torch
    L = lbmlib
    theta = inputs.xavier_params(77, s_df=1e-3, bias_scale=0.1)
    params = torch.from_numpy(theta).to(cuda)
    packed = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=cuda)
    L.gnn_pack(params, packed)
    cases = [(1, 80, 96, 0.8), (2, 128, 128, 0.65)]   # the second is exactly the limit
    assert 2 * 128 * 128 == L.LBM_STEP_GNN_NOALLOC_MAX_NODES
    for (nb, ny, nx, tau) in cases:
        f = _state(nb, ny, nx, seed=nx + ny)
        fin, _ = to_dev(f, cuda)
        s = L.shape(nx, ny, nb)
        ref = torch.full_like(fin, float("nan"))
        ws = torch.empty(L.gnn_step_workspace_bytes(s), dtype=torch.uint8, device=cuda)
        L.lbm_step_gnn(fin, ref, s, tau, None, packed, None, ws)
        got = torch.full_like(fin, float("nan"))
        tot = torch.zeros(5, dtype=torch.float64, device=cuda)
        L.lbm_step_gnn_noalloc(fin, got, s, tau, None, packed, tot)
        assert L.lbm_get_status() == 0
        assert torch.isfinite(got).all()
        assert torch.allclose(got, ref, rtol=1e-6, atol=0)
        assert tot[0].item() > 0


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
