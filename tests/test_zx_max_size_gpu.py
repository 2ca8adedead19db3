"""A BGK step on a stack larger than 2^31 nodes (65,536 x 32,769 nodes,
77 GB per population buffer), so that every node index, plane offset and
launch size takes its 64-bit path.  The bounds-checked build runs first (an
index out of range would raise the status word's bounds bit instead of
being read); then the regular build.  Checked at sampled nodes around index
2^31, the lattice corners and both wraps against the oracle's BGK step of
each node's 3 x 3 neighbourhood (the step reads nothing further), 1e-6
relative per population, and the FP64 totals (mass = sum of rho to 1e-9)."""
import numpy as np
import pytest

from oracle import lbm

pytestmark = pytest.mark.gpu

NX, NY = 65536, 32769          # N = 2,147,549,184 > 2^31
TAU = 0.8
SAMPLES = [(0, 32768), (1, 32768), (65535, 32767), (65535, 32768), (0, 0), (65535, 0),
           (32768, 16384), (12345, 32767), (4, 32768)]


def _patch(f, x, y):
    """[9, 3, 3] periodic neighbourhood of (x, y) from the device state."""
    import torch
    xs = torch.tensor([(x + d) % NX for d in (-1, 0, 1)], device=f.device)
    ys = torch.tensor([(y + d) % NY for d in (-1, 0, 1)], device=f.device)
    idx = (ys[:, None] * NX + xs[None, :]).reshape(-1)
    return f.view(9, -1)[:, idx].reshape(9, 3, 3).double().cpu().numpy()


def _run(L, f_in, f_out, tot):
    import torch
    s = L.shape(NX, NY)
    k = 2 * np.pi / NX
    L.lbm_init_tgv(f_in, s, 1.0, 0.05, k, 2 * np.pi / NY, False)
    L.lbm_step_bgk(f_in, f_out, None, s, TAU, totals=tot)
    torch.cuda.synchronize()
    return L.lbm_get_status()


def test_bgk_step_beyond_2_31_nodes(lbmlib, cuda):
    import torch
    from paper_2504_14494_gb300 import build, lib as L
    n = NX * NY
    assert n > 2 ** 31
    torch.cuda.empty_cache()  # blocks cached by earlier tests
    free, _ = torch.cuda.mem_get_info()
    if free < 2 * 9 * n * 4 + (4 << 30):
        pytest.skip("needs 160 GB of free device memory")
    f_in = torch.empty(9 * n, dtype=torch.float32, device=cuda)
    f_out = torch.empty_like(f_in)
    tot = torch.zeros(5, dtype=torch.float64, device=cuda)
    regular = L._lib
    try:
        L._lib = None
        L.load(build.build(checked=True))
        assert _run(L, f_in, f_out, tot) == L.LBM_OK  # LBM_ERR_BOUNDS: an index out of range
    finally:
        L._lib = regular
    assert _run(L, f_in, f_out, tot) == L.LBM_OK
    for x, y in SAMPLES:
        want = lbm.bgk_step(_patch(f_in, x, y), TAU)[:, 1, 1]
        got = f_out.view(9, -1)[:, y * NX + x].double().cpu().numpy()
        assert np.allclose(got, want, rtol=1e-6, atol=0), (x, y, got, want)
    t = tot.cpu().numpy()
    planes = f_out.view(9, -1)
    rho_sum = sum(float(planes[q, i:i + (1 << 27)].double().sum().item())
                  for q in range(9) for i in range(0, n, 1 << 27))
    assert abs(t[0] - rho_sum) <= 1e-9 * rho_sum
    assert t[4] == 0.0
    del f_in, f_out
    torch.cuda.empty_cache()


def test_gnn_step_at_16384_squared(lbmlib, cuda):
    """lbm_step_gnn on one 16,384^2 lattice (268 M nodes: 137 GB of
    workspace, plane offsets beyond 2^35 bytes), bounds-checked build first,
    then the regular build: sampled nodes (the last rows and columns
    included) against the oracle's GNN step of the 13 x 13 periodic patch
    around each (streaming plus two message-passing hops reach 3 nodes), at
    the tolerance of the 1024^2 sampled test."""
    import torch
    from oracle import gnn
    from paper_2504_14494_gb300 import build, inputs, lib as L
    from gpu_util import rel_l2
    n = 16384
    torch.cuda.empty_cache()
    s = L.shape(n, n)
    need = 2 * 9 * n * n * 4 + L.gnn_step_workspace_bytes(s) + (4 << 30)
    if torch.cuda.mem_get_info()[0] < need:
        pytest.skip("needs 162 GB of free device memory")
    k = 2 * np.pi / n
    f = torch.empty(9 * n * n, device=cuda)
    out = torch.empty_like(f)
    ws = torch.empty(L.gnn_step_workspace_bytes(s), dtype=torch.uint8, device=cuda)
    theta = inputs.xavier_params(53, s_df=1e-2, bias_scale=0.1)
    params = torch.from_numpy(theta).to(cuda)

    def run():
        pk = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=cuda)
        L.gnn_pack(params, pk)
        L.lbm_init_tgv(f, s, 1.0, 0.05, k, k, False)
        L.lbm_step_gnn(f, out, s, 0.65, None, pk, None, ws)
        torch.cuda.synchronize()
        return L.lbm_get_status()

    regular = L._lib
    try:
        L._lib = None
        L.load(build.build(checked=True))
        assert run() == L.LBM_OK  # LBM_ERR_BOUNDS: an index out of range
    finally:
        L._lib = regular
    assert run() == L.LBM_OK
    rng = np.random.default_rng(3)
    pts = [(int(a), int(b)) for a, b in zip(rng.integers(0, n, 24), rng.integers(0, n, 24))]
    pts += [(0, 0), (n - 1, n - 1), (n - 1, 0), (0, n - 1), (n // 2, n - 1)]
    F = f.view(9, n, n)
    got, ref, bgk = [], [], []
    for (x, y) in pts:
        xs = torch.tensor((np.arange(x - 6, x + 7)) % n, device=cuda)
        ys = torch.tensor((np.arange(y - 6, y + 7)) % n, device=cuda)
        patch = F[:, ys[:, None], xs[None, :]].double().cpu().numpy()
        ref.append(gnn.gnn_step(patch, theta, 0.65)[:, 6, 6])
        bgk.append(lbm.bgk_step(patch, 0.65)[:, 6, 6])
        got.append(out.view(9, n, n)[:, y, x].double().cpu().numpy())
    got, ref, bgk = np.array(got), np.array(ref), np.array(bgk)
    assert rel_l2(got - bgk, ref - bgk) <= 3e-2
    del f, out, ws
    torch.cuda.empty_cache()
