"""Batched run of uneven lattices (one CUDA graph launch per call) against
per-lattice runs of the same kernels and against the oracle.

The per-node arithmetic of the batched kernels is that of the single-lattice
kernels (each tensor-core row depends only on its own node), so each lattice
of the batch must equal its own single-lattice run to FP32 rounding
(<= 1e-6 relative; identical in practice)."""
import json
import os

import numpy as np
import pytest

from oracle import lbm
from paper_2504_14494_gb300 import inputs

pytestmark = pytest.mark.gpu

LATTICES = [(8, 8, 0, 0.8), (13, 7, 1, 0.7), (32, 32, 0, 0.55), (5, 9, 1, 0.9),
            (64, 48, 0, 1.3), (20, 20, 1, 0.62), (1, 1, 0, 0.8), (3, 130, 1, 0.75)]


def _prm(i, nx, ny):
    return (1.0, 0.02 + 0.01 * (i % 5), 2 * np.pi / nx, 2 * np.pi / ny)


def test_batched_run_equals_per_lattice_runs(lbmlib, cuda, tmp_path):
    import torch
    L = lbmlib
    theta = inputs.xavier_params(17, s_df=1e-3, bias_scale=0.1)
    params = torch.from_numpy(theta).to(cuda)
    packed = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=cuda)
    L.gnn_pack(params, packed)
    plan = L.lbm_batch_plan_create(LATTICES)
    try:
        n = L.lbm_batch_nodes(plan)
        assert n == sum(a * b for a, b, _, _ in LATTICES)
        off = L.lbm_batch_offsets(plan, len(LATTICES))
        # BGK group first, then GNN group, input order inside each
        order = [i for i, l in enumerate(LATTICES) if l[2] == 0] + \
                [i for i, l in enumerate(LATTICES) if l[2] == 1]
        acc = 0
        for i in order:
            assert off[i] == acc
            acc += LATTICES[i][0] * LATTICES[i][1]
        prm = np.array([_prm(i, l[0], l[1]) for i, l in enumerate(LATTICES)])
        f0 = torch.empty(9 * n, device=cuda)
        L.lbm_batch_init_tgv(plan, f0, prm, False)
        f1, f2 = torch.empty_like(f0), torch.empty_like(f0)
        ws = torch.empty(max(L.lbm_batch_workspace_bytes(plan), 16), dtype=torch.uint8, device=cuda)
        steps = 3
        L.lbm_batch_run(plan, f0, f1, f2, steps, packed, ws)
        # replay of the recorded graph gives the same result
        again = torch.empty_like(f0)
        L.lbm_batch_run(plan, f0, again, f2, steps, packed, ws)
        assert L.lbm_get_status() == 0
        assert torch.equal(f1, again)
        F0 = f0.view(9, n)
        F1 = f1.view(9, n)
        for i, (nx, ny, col, tau) in enumerate(LATTICES):
            m = nx * ny
            init = F0[:, off[i]:off[i] + m].contiguous()
            ref_tgv = lbm.tgv_init(nx, ny, *prm[i]).reshape(9, -1)
            assert np.all(np.abs(init.cpu().numpy() - ref_tgv) <= 1.2e-7 * np.abs(ref_tgv))
            a = init.reshape(-1).clone()
            b = torch.empty_like(a)
            s = L.shape(nx, ny)
            for _ in range(steps):
                if col == 0:
                    L.lbm_step_bgk(a, b, None, s, tau)
                else:
                    w = torch.empty(L.gnn_step_workspace_bytes(s), dtype=torch.uint8, device=cuda)
                    L.lbm_step_gnn(a, b, s, tau, None, packed, None, w)
                a, b = b, a
            got = F1[:, off[i]:off[i] + m]
            ref = a.view(9, m)
            assert torch.allclose(got, ref, rtol=1e-6, atol=0), (i, nx, ny, col)
            if col == 0:
                o = lbm.bgk_run(ref_tgv.reshape(9, ny, nx), tau, steps).reshape(9, -1)
                assert np.allclose(got.double().cpu().numpy(), o, rtol=3e-6, atol=0)
        # another step count re-records the graph
        L.lbm_batch_run(plan, f0, f1, f2, 1, packed, ws)
        ref1 = torch.empty_like(f0)
        L.lbm_batch_run(plan, f0, ref1, f2, 2, packed, ws)
        L.lbm_batch_run(plan, ref1, f2, again, 0, packed, ws)   # steps = 0 copies
        assert torch.equal(ref1, f2)
        assert L.lbm_get_status() == 0
        path = tmp_path / "tune.json"
        L.lbm_autotune_save(path)
        tuned = json.loads(path.read_text())
        assert any(k.startswith("bgk_batch_tile/") for k in tuned)
        assert any(k.startswith("gnn_step_table/") for k in tuned)
        L.lbm_autotune_load(path)
    finally:
        L.lbm_batch_plan_destroy(plan)


@pytest.mark.parametrize("variant", [0, 1])
def test_stack_and_table_geometry_agree_bitwise(lbmlib, cuda, variant):
    """Lattices stepped alone by lbm_step_gnn (stack geometry, positions by
    multiply-high division) and together by the batched run (table geometry,
    lattice found by binary search): the same arithmetic in the same order,
    so bitwise equal.  Variant 1 (MLP only) takes the short path of both:
    no edge terms, no inner round."""
    import torch
    L = lbmlib
    lat = [(128, 6, 1, 0.7), (256, 3, 1, 0.62), (384, 2, 1, 0.9), (64, 8, 1, 0.75),
           (32, 4, 1, 0.8), (96, 12, 1, 0.66)]
    theta = inputs.xavier_params(19, s_df=1e-2, bias_scale=0.1, variant=variant)
    params = torch.from_numpy(theta).to(cuda)
    packed = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=cuda)
    L.gnn_pack(params, packed)
    plan = L.lbm_batch_plan_create(lat)
    try:
        n = L.lbm_batch_nodes(plan)
        off = L.lbm_batch_offsets(plan, len(lat))
        prm = np.array([_prm(i, l[0], l[1]) for i, l in enumerate(lat)])
        f0 = torch.empty(9 * n, device=cuda)
        L.lbm_batch_init_tgv(plan, f0, prm, False)
        g = torch.Generator(device=cuda)
        g.manual_seed(11)
        f0.mul_(1 + 2e-2 * (2 * torch.rand(f0.shape, generator=g, device=cuda) - 1))
        f1, f2 = torch.empty_like(f0), torch.empty_like(f0)
        ws = torch.empty(L.lbm_batch_workspace_bytes(plan), dtype=torch.uint8, device=cuda)
        L.lbm_batch_run(plan, f0, f1, f2, 1, packed, ws)
        for i, (nx, ny, _, tau) in enumerate(lat):
            m = nx * ny
            a = f0.view(9, n)[:, off[i]:off[i] + m].contiguous().reshape(-1)
            b = torch.empty_like(a)
            s = L.shape(nx, ny)
            w = torch.empty(L.gnn_step_workspace_bytes(s), dtype=torch.uint8, device=cuda)
            L.lbm_step_gnn(a, b, s, tau, None, packed, None, w)
            assert torch.equal(f1.view(9, n)[:, off[i]:off[i] + m], b.view(9, m)), (nx, ny)
        assert L.lbm_get_status() == 0
    finally:
        L.lbm_batch_plan_destroy(plan)


def test_batch_plan_argument_checks(lbmlib):
    L = lbmlib
    with pytest.raises(L.LbmError) as e:
        L.lbm_batch_plan_create([(8, 8, 0, 0.5)])
    assert e.value.code == -4
    with pytest.raises(L.LbmError) as e:
        L.lbm_batch_plan_create([(0, 8, 0, 0.8)])
    assert e.value.code == -3
    with pytest.raises(L.LbmError) as e:
        L.lbm_batch_plan_create([(8, 8, 7, 0.8)])
    assert e.value.code == -1
    with pytest.raises(L.LbmError) as e:  # a lattice of 2^31 nodes
        L.lbm_batch_plan_create([(8, 8, 0, 0.8), (65536, 32768, 1, 0.8)])
    assert e.value.code == L.LBM_ERR_SIZE


def test_every_bgk_tile_shape_gives_the_same_bits(lbmlib, cuda, tmp_path):
    """Each tile shape the autotuner can choose for the batched BGK kernel
    (threads per block x nodes per thread, forced through a loaded cache)
    schedules the same per-node arithmetic: identical results."""
    import torch
    L = lbmlib
    lat = [(8, 8, 0, 0.8), (33, 7, 0, 0.7), (130, 5, 0, 0.55), (1, 1, 0, 0.9), (64, 40, 0, 1.1)]
    nodes = sum(a * b for a, b, _, _ in lat)
    sms = torch.cuda.get_device_properties(cuda).multi_processor_count
    bucket = int(np.floor(np.log2(nodes)))
    out = None
    for tile in (1281, 1282, 1284, 2561, 2562, 2564, 5121, 5122):
        path = tmp_path / f"tile{tile}.json"
        path.write_text(json.dumps({f"bgk_batch_tile/sm{sms}/n2^{bucket}": tile}))
        L.lbm_autotune_load(path)
        plan = L.lbm_batch_plan_create(lat)
        try:
            n = L.lbm_batch_nodes(plan)
            prm = np.array([_prm(i, l[0], l[1]) for i, l in enumerate(lat)])
            f0 = torch.empty(9 * n, device=cuda)
            L.lbm_batch_init_tgv(plan, f0, prm, False)
            f1, f2 = torch.empty_like(f0), torch.empty_like(f0)
            L.lbm_batch_run(plan, f0, f1, f2, 3, None, None)
            assert L.lbm_get_status() == 0
            if out is None:
                out = f1.clone()
            else:
                assert torch.equal(out, f1), tile
        finally:
            L.lbm_batch_plan_destroy(plan)


def test_serving_batch_of_512_lattices_sampled_against_the_oracle(lbmlib, cuda):
    """The 512-lattice serving workload as the benchmark builds it (sides
    log-uniform in [32, 1024], Re ~ U[100, 5000], u0 ~ U[0.01, 0.08], seed 7;
    half BGK, half GNN-LBM with a message-passing conserving network), one
    batched step: sampled nodes of the largest, the smallest and 10 more GNN
    lattices (corners, edges, interior) against the oracle's GNN step of the
    13 x 13 periodic patch around each, and of 8 BGK lattices against the
    oracle's BGK step of the 3 x 3 patch.  Tolerances as the single-lattice
    GNN-LBM step tests (correction rel L2 <= 3e-2, per-population bound) and
    1e-6 per population for BGK."""
    import torch
    from oracle import gnn
    from gpu_util import rel_l2
    L = lbmlib
    draws = inputs.batch_lattices(512, 7, 32, 1024, 100.0, 5000.0)
    lat = [(d["side"], d["side"], 1 if d["gnn"] else 0, 0.5 + 3.0 * d["nu"]) for d in draws]
    theta = inputs.xavier_params(0, s_df=1e-2, bias_scale=0.1, variant=2)
    packed = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=cuda)
    L.gnn_pack(torch.from_numpy(theta).to(cuda), packed)
    plan = L.lbm_batch_plan_create(lat)
    try:
        n = L.lbm_batch_nodes(plan)
        off = L.lbm_batch_offsets(plan, len(lat))
        prm = np.array([(1.0, d["u0"], 2 * np.pi / d["side"], 2 * np.pi / d["side"])
                        for d in draws])
        f0 = torch.empty(9 * n, device=cuda)
        L.lbm_batch_init_tgv(plan, f0, prm, True)
        g = torch.Generator(device=cuda)
        g.manual_seed(5)
        f0.mul_(1 + 1e-2 * (2 * torch.rand(f0.shape, generator=g, device=cuda) - 1))
        f1 = torch.empty_like(f0)
        ws = torch.empty(L.lbm_batch_workspace_bytes(plan), dtype=torch.uint8, device=cuda)
        L.lbm_batch_run(plan, f0, f1, None, 1, packed, ws)
        assert L.lbm_get_status() == 0
        F0, F1 = f0.view(9, n), f1.view(9, n)
        rng = np.random.default_rng(3)
        gnn_ids = [i for i, d in enumerate(draws) if d["gnn"]]
        bgk_ids = [i for i, d in enumerate(draws) if not d["gnn"]]
        by_size = sorted(gnn_ids, key=lambda i: draws[i]["side"])
        pick = [by_size[-1], by_size[0]] + [int(i) for i in rng.choice(by_size[1:-1], 10, False)]
        got, ref, bgk = [], [], []
        for i in pick:
            side, tau = draws[i]["side"], lat[i][3]
            lf0 = F0[:, off[i]:off[i] + side * side].view(9, side, side)
            lf1 = F1[:, off[i]:off[i] + side * side].view(9, side, side)
            pts = [(0, 0), (side - 1, side - 1), (0, side // 2)]
            pts.append(tuple(int(v) for v in rng.integers(0, side, 2)))
            for (y, x) in pts:
                ys = [(y + d) % side for d in range(-6, 7)]
                xs = [(x + d) % side for d in range(-6, 7)]
                patch = lf0[:, ys][:, :, xs].double().cpu().numpy()
                ref.append(gnn.gnn_step(patch, theta, tau)[:, 6, 6])
                bgk.append(lbm.bgk_step(patch, tau)[:, 6, 6])
                got.append(lf1[:, y, x].double().cpu().numpy())
        got, ref, bgk = np.array(got), np.array(ref), np.array(bgk)
        e_corr = rel_l2(got - bgk, ref - bgk)
        e_f = np.max(np.abs(got - ref) - 1e-6 * np.abs(ref)) / np.max(np.abs(ref - bgk))
        print(f"{len(got)} GNN nodes of {len(pick)} lattices: correction rel L2 {e_corr:.2e}, "
              f"max err / max correction {e_f:.2e}")
        assert e_corr <= 3e-2 and e_f <= 5e-2, (e_corr, e_f)
        for i in [int(v) for v in rng.choice(bgk_ids, 8, False)]:
            side, tau = draws[i]["side"], lat[i][3]
            lf0 = F0[:, off[i]:off[i] + side * side].view(9, side, side)
            lf1 = F1[:, off[i]:off[i] + side * side].view(9, side, side)
            for (y, x) in [(0, 0), (side - 1, 3), tuple(int(v) for v in rng.integers(0, side, 2))]:
                ys = [(y + d) % side for d in (-1, 0, 1)]
                xs = [(x + d) % side for d in (-1, 0, 1)]
                patch = lf0[:, ys][:, :, xs].double().cpu().numpy()
                want = lbm.bgk_step(patch, tau)[:, 1, 1]
                have = lf1[:, y, x].double().cpu().numpy()
                assert np.all(np.abs(have - want) <= 1e-6 * np.abs(want)), (i, y, x)
    finally:
        L.lbm_batch_plan_destroy(plan)
