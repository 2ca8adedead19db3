"""Parity of the CUDA BGK path (through the C ABI) with the FP64 oracle.

Tolerances (stated):
  * one step from an identical FP32 input: |f_gpu - f_oracle| <= 1e-6 |f_oracle|
    per element (the kernel computes in FP32; its rounding error is a few ulp);
  * 1000 steps of the 64^2 TGV: relative L2 of the velocity difference <= 1e-4,
    kinetic energy within 1e-3 relative, FP32 mass drift <= 1e-5 relative;
  * initial state: FP64 arithmetic rounded once to FP32 (<= 1 ulp);
  * FP64 totals of a state: within FP32 input rounding of the oracle's.
"""
import json
import os

import numpy as np
import pytest

from oracle import lbm
from paper_2504_14494_gb300 import inputs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _to_dev(a, dev, plane_stride=0):
    import torch
    a = np.ascontiguousarray(a, dtype=np.float32)
    q = a.shape[0]
    n = a[0].size
    ps = plane_stride or n
    buf = torch.zeros(q * ps, dtype=torch.float32, device=dev)
    view = buf.view(q, ps)[:, :n]
    view.copy_(torch.from_numpy(a.reshape(q, n)))
    return buf, ps


def _from_dev(buf, shape, ps):
    q = shape[0]
    n = int(np.prod(shape[1:]))
    return buf.view(q, ps)[:, :n].cpu().numpy().reshape(shape).astype(np.float64)


def _input(nb, ny, nx, seed, u0=0.05):
    f = np.stack([lbm.tgv_init(nx, ny, 1.0, u0, 2 * np.pi / nx, 2 * np.pi / ny)] * nb, axis=1)
    f = f * inputs.perturbation(f.shape, seed, 1e-2)
    return f.astype(np.float32)           # (9, nb, ny, nx)


def _oracle_step(f32, tau):
    taus = np.broadcast_to(np.asarray(tau, np.float64), (f32.shape[1],))
    return np.stack([lbm.bgk_step(f32[:, b].astype(np.float64), taus[b])
                     for b in range(f32.shape[1])], axis=1)


SHAPES = [(1, 64, 64), (1, 1, 1), (1, 2, 2), (1, 3, 3), (1, 3, 5), (1, 7, 132), (3, 20, 36),
          (2, 16, 260), (1, 9, 4), (4, 5, 8)]


@pytest.mark.parametrize("nb,ny,nx", SHAPES)
def test_one_step_matches_oracle(lbmlib, cuda, nb, ny, nx):
    import torch
    L = lbmlib
    f = _input(nb, ny, nx, seed=nx * 131 + ny)
    din, ps = _to_dev(f, cuda)
    dout = torch.full_like(din, float("nan"))
    s = L.shape(nx, ny, nb)
    L.lbm_step_bgk(din, dout, None, s, 0.8, nsteps=1)
    torch.cuda.synchronize()
    got = _from_dev(dout, f.shape, ps)
    ref = _oracle_step(f, 0.8)
    assert np.all(np.abs(got - ref) <= 1e-6 * np.abs(ref)), np.max(np.abs(got - ref) / np.abs(ref))
    assert L.lbm_get_status() == 0


def test_per_lattice_tau_and_padded_stride(lbmlib, cuda):
    import torch
    L = lbmlib
    nb, ny, nx = 3, 12, 16
    f = _input(nb, ny, nx, seed=3)
    ps = nb * ny * nx + 52          # padded planes (multiple of 4)
    din, _ = _to_dev(f, cuda, plane_stride=ps)
    dout = torch.zeros_like(din)
    taus = np.array([0.55, 0.8, 1.7], np.float32)
    dt = torch.from_numpy(taus).to(cuda)
    L.lbm_step_bgk(din, dout, None, L.shape(nx, ny, nb, ps), 9.0, taus=dt, nsteps=1)
    got = _from_dev(dout, f.shape, ps)
    ref = _oracle_step(f, taus.astype(np.float64))
    assert np.all(np.abs(got - ref) <= 1e-6 * np.abs(ref))
    # padding is untouched
    assert torch.count_nonzero(dout.view(9, ps)[:, nb * ny * nx:]) == 0


def test_unaligned_base_takes_general_path(lbmlib, cuda):
    import torch
    L = lbmlib
    f = _input(1, 8, 16, seed=4)
    n = f[0].size
    big = torch.zeros(9 * n + 1, dtype=torch.float32, device=cuda)
    big[1:].copy_(torch.from_numpy(f.reshape(-1)))
    out = torch.zeros(9 * n + 1, dtype=torch.float32, device=cuda)
    L.lbm_step_bgk(big.data_ptr() + 4, out.data_ptr() + 4, None, L.shape(16, 8), 0.8)
    got = out[1:].cpu().numpy().reshape(f.shape).astype(np.float64)
    ref = _oracle_step(f, 0.8)
    assert np.all(np.abs(got - ref) <= 1e-6 * np.abs(ref))


def test_multi_step_pingpong_and_totals(lbmlib, cuda):
    """nsteps = 0..5 with ping-pong buffers land in f_out; the FP64 totals of
    the final state match the oracle's totals of the GPU state."""
    import torch
    L = lbmlib
    f = _input(2, 16, 24, seed=5)
    din, ps = _to_dev(f, cuda)
    for nsteps in range(6):
        dout = torch.zeros_like(din)
        tmp = torch.zeros_like(din)
        tot = torch.zeros(5, dtype=torch.float64, device=cuda)
        L.lbm_step_bgk(din, dout, tmp, L.shape(24, 16, 2), 0.7, nsteps=nsteps, totals=tot)
        got = _from_dev(dout, f.shape, ps)
        ref = f.astype(np.float64)
        for _ in range(nsteps):
            ref = _oracle_step(ref.astype(np.float64), 0.7)
        assert np.allclose(got, ref, rtol=1e-5 * max(nsteps, 1), atol=0)
        t_ref = sum(lbm.totals(got[:, b]) for b in range(2))
        t = tot.cpu().numpy()
        assert abs(t[0] - t_ref[0]) <= 1e-12 * t_ref[0]
        assert abs(t[1] - t_ref[1]) <= 1e-9 and abs(t[2] - t_ref[2]) <= 1e-9
        assert abs(t[3] - t_ref[3]) <= 1e-6 * t_ref[3]
        assert t[4] == 0


def test_tgv_init_matches_oracle(lbmlib, cuda):
    import torch
    L = lbmlib
    for pc in (False, True):
        nb, ny, nx = 2, 24, 40
        f = torch.zeros(9 * nb * ny * nx, dtype=torch.float32, device=cuda)
        L.lbm_init_tgv(f, L.shape(nx, ny, nb), 1.0, 0.05, 2 * np.pi / nx, 2 * np.pi / ny, pc)
        got = f.view(9, nb, ny, nx).cpu().numpy()
        ref = lbm.tgv_init(nx, ny, 1.0, 0.05, 2 * np.pi / nx, 2 * np.pi / ny, pc)
        for b in range(nb):
            assert np.all(np.abs(got[:, b] - ref) <= 6e-8 * np.abs(ref))


def test_moments_match_oracle(lbmlib, cuda):
    import torch
    L = lbmlib
    f = _input(2, 10, 12, seed=6)
    din, ps = _to_dev(f, cuda)
    n = f[0].size
    rho = torch.zeros(n, device=cuda)
    ux = torch.zeros(n, device=cuda)
    uy = torch.zeros(n, device=cuda)
    tot = torch.zeros(5, dtype=torch.float64, device=cuda)
    L.lbm_moments(din, L.shape(12, 10, 2), rho, ux, uy, tot)
    r, x, y = lbm.moments(f.astype(np.float64).reshape(9, -1))
    assert np.allclose(rho.cpu().numpy(), r, rtol=3e-7, atol=0)
    assert np.allclose(ux.cpu().numpy(), x, rtol=0, atol=3e-8)
    assert np.allclose(uy.cpu().numpy(), y, rtol=0, atol=3e-8)
    t_ref = lbm.totals(f.astype(np.float64).reshape(9, 1, -1))
    t = tot.cpu().numpy()
    assert abs(t[0] - t_ref[0]) <= 1e-6 * t_ref[0]
    assert abs(t[3] - t_ref[3]) <= 1e-5 * t_ref[3]


def test_totals_accuracy_at_scale(lbmlib, cuda):
    """The totals are summed as FP32 pairs (error-free TwoSum) and combined in
    FP64 once per warp: on 3 x 256 x 320 nodes of a perturbed state with a
    few NaN nodes and one strongly non-equilibrium patch, mass within 1e-13
    relative of the FP64 sum of the same FP32 values, momentum within
    1e-13 of sum |f|, energy within 1e-6 relative, NaN nodes counted."""
    import torch
    L = lbmlib
    nb, ny, nx = 3, 256, 320
    f = _input(nb, ny, nx, seed=11, u0=0.08)
    f[:, 1, 10:20, 30:50] *= inputs.perturbation(f[:, 1, 10:20, 30:50].shape, 12, 0.9)
    f[3, 2, 7, 9] = np.nan
    f[0, 0, 100, 1] = np.inf
    din, _ = _to_dev(f, cuda)
    tot = torch.zeros(5, dtype=torch.float64, device=cuda)
    L.lbm_moments(din, L.shape(nx, ny, nb), None, None, None, tot)
    t = tot.cpu().numpy()
    assert L.lbm_get_status() == -7          # LBM_ERR_NONFINITE, cleared by the read
    t_ref = sum(lbm.totals(f[:, b].astype(np.float64)) for b in range(nb))
    ok = np.all(np.isfinite(f), axis=0)
    absum = np.sum(np.abs(np.where(ok[None], f.astype(np.float64), 0.0)))
    assert t[4] == t_ref[4] == 2
    assert abs(t[0] - t_ref[0]) <= 1e-13 * t_ref[0], (t[0], t_ref[0])
    assert abs(t[1] - t_ref[1]) <= 1e-13 * absum, (t[1], t_ref[1])
    assert abs(t[2] - t_ref[2]) <= 1e-13 * absum, (t[2], t_ref[2])
    assert abs(t[3] - t_ref[3]) <= 1e-6 * t_ref[3], (t[3], t_ref[3])


def test_tgv64_1000_steps_matches_oracle(lbmlib, cuda):
    """The 64^2 TGV workload (tau=0.8, u0=0.01, 1000 steps): velocity field,
    L2 error vs the closed form, energy and mass drift against the FP64 oracle
    values stored by tests/golden/make_golden.py."""
    import torch
    L = lbmlib
    with open(os.path.join(GOLDEN, "tgv64_bgk.json")) as fh:
        gold = json.load(fh)
    n, u0, tau, steps = gold["n"], gold["u0"], gold["tau"], gold["steps"]
    k = 2 * np.pi / n
    s = L.shape(n, n)
    f0 = torch.zeros(9 * n * n, device=cuda)
    L.lbm_init_tgv(f0, s, 1.0, u0, k, k, False)
    f1, tmp = torch.zeros_like(f0), torch.zeros_like(f0)
    tot = torch.zeros(5, dtype=torch.float64, device=cuda)
    L.lbm_step_bgk(f0, f1, tmp, s, tau, nsteps=steps, totals=tot)
    rho, ux, uy = (torch.zeros(n * n, device=cuda) for _ in range(3))
    L.lbm_moments(f1, s, rho, ux, uy)
    assert L.lbm_get_status() == 0
    ux, uy = ux.cpu().numpy().reshape(n, n), uy.cpu().numpy().reshape(n, n)
    ref = lbm.bgk_run(lbm.tgv_init(n, n, 1.0, u0, k, k), tau, steps)
    _, rx, ry = lbm.moments(ref)
    diff = np.sqrt(np.sum((ux - rx) ** 2 + (uy - ry) ** 2) / np.sum(rx ** 2 + ry ** 2))
    assert diff <= 1e-4, diff
    err = lbm.velocity_l2_error(ux, uy, *lbm.tgv_analytic_velocity(n, n, u0, k, k, tau, steps))
    assert abs(err - gold["l2_error"]) <= 1e-4
    t = tot.cpu().numpy()
    assert abs(t[3] - gold["totals"][3]) <= 1e-3 * gold["totals"][3]
    assert abs(t[0] - gold["totals0"][0]) <= 1e-5 * gold["totals0"][0]


def test_nonfinite_input_is_flagged(lbmlib, cuda):
    """A NaN population (made on the host) is counted in the totals and raises
    LBM_ERR_NONFINITE through the status word; the GPU is not faulted."""
    import torch
    L = lbmlib
    f = _input(1, 8, 8, seed=7)
    f[3, 0, 2, 5] = np.nan
    din, _ = _to_dev(f, cuda)
    dout = torch.zeros_like(din)
    tot = torch.zeros(5, dtype=torch.float64, device=cuda)
    L.lbm_step_bgk(din, dout, None, L.shape(8, 8), 0.8, totals=tot)
    assert L.lbm_get_status() == -7
    assert tot[4].item() >= 1
    assert L.lbm_get_status() == 0          # cleared by the read


def test_full_size_4096_sampled(lbmlib, cuda):
    """At the 4096^2 bandwidth workload, in the launch configuration the
    benchmark times: one step from the TGV state, checked at 4096 sampled
    nodes (and every node of the four edge rows/columns) against the oracle
    collision of the pulled populations."""
    import torch
    L = lbmlib
    n = 4096
    s = L.shape(n, n)
    f0 = torch.empty(9 * n * n, device=cuda)
    L.lbm_init_tgv(f0, s, 1.0, 0.05, 2 * np.pi / n, 2 * np.pi / n, False)
    # perturb so that every node differs from equilibrium
    g = torch.Generator(device=cuda)
    g.manual_seed(11)
    f0.mul_(1 + 1e-2 * (2 * torch.rand(f0.shape, generator=g, device=cuda) - 1))
    f1 = torch.empty_like(f0)
    L.lbm_step_bgk(f0, f1, None, s, 0.5614, nsteps=1)
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.integers(0, n, 4096), np.arange(n), np.arange(n), np.zeros(n, int), np.full(n, n - 1)])
    ys = np.concatenate([rng.integers(0, n, 4096), np.zeros(n, int), np.full(n, n - 1), np.arange(n), np.arange(n)])
    F0 = f0.view(9, n, n)
    pulled = np.empty((9, 1, xs.size))
    for q in range(9):
        sx = torch.from_numpy((xs - lbm.E[q, 0]) % n).to(cuda)
        sy = torch.from_numpy((ys - lbm.E[q, 1]) % n).to(cuda)
        pulled[q, 0] = F0[q][sy, sx].double().cpu().numpy()
    ref = lbm.bgk_collide(pulled, 0.5614)[:, 0]
    got = f1.view(9, n, n)[:, torch.from_numpy(ys).to(cuda), torch.from_numpy(xs).to(cuda)].double().cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-6 * np.abs(ref))


def test_bounded_wait_reports_timeout(lbmlib, cuda):
    """A device wait on a barrier nothing arrives on gives up after its
    budget (~1 ms here) and reports LBM_ERR_TIMEOUT through the status word;
    the context stays usable (a BGK step afterwards is correct)."""
    import torch
    L = lbmlib
    assert L.lbm_get_status() == 0
    L.lbm_selftest_wait_timeout(2_000_000)
    assert L.lbm_get_status() == -8
    assert L.lbm_get_status() == 0
    f = _input(1, 8, 8, seed=12)
    din, _ = _to_dev(f, cuda)
    dout = torch.zeros_like(din)
    L.lbm_step_bgk(din, dout, None, L.shape(8, 8), 0.8)
    ref = _oracle_step(f, 0.8)
    assert np.all(np.abs(_from_dev(dout, f.shape, din.numel() // 9) - ref) <= 1e-6 * np.abs(ref))


@pytest.mark.parametrize("nb,ny,nx,nsteps,per_lattice", [
    (1, 64, 96, 1, False), (1, 64, 96, 3, False), (3, 20, 36, 2, True), (2, 5, 30, 1, True),
    (1, 3, 8, 4, False), (5, 7, 12, 1, False)])
def test_host_buffer_step_equals_device_step(lbmlib, cuda, nb, ny, nx, nsteps, per_lattice):
    """lbm_step_bgk_host (state in host memory, chunked copy overlapped with
    the first step) gives bitwise the state and totals of lbm_step_bgk on the
    device copy, for pinned and pageable host memory."""
    import torch
    L = lbmlib
    s = L.shape(nx, ny, nb)
    f = _input(nb, ny, nx, seed=21)
    taus = np.linspace(0.6, 0.9, nb).astype(np.float32)
    din, _ = _to_dev(f, cuda)
    dout, tmp = torch.zeros_like(din), torch.zeros_like(din)
    tot = torch.zeros(5, dtype=torch.float64, device=cuda)
    dtaus = torch.from_numpy(taus).to(cuda) if per_lattice else None
    L.lbm_step_bgk(din, dout, tmp, s, 0.7, taus=dtaus, nsteps=nsteps, totals=tot)
    want, want_tot = dout.cpu(), tot.cpu()
    ws = torch.empty(L.lbm_host_workspace_bytes(s), dtype=torch.uint8, device=cuda)
    for pinned in (True, False):
        h_in = torch.from_numpy(f.reshape(-1).copy())
        h_out = torch.full_like(h_in, -1.0)
        h_tot = torch.zeros(5, dtype=torch.float64)
        h_taus = torch.from_numpy(taus.copy()) if per_lattice else None
        if pinned:
            h_in, h_out, h_tot = h_in.pin_memory(), h_out.pin_memory(), h_tot.pin_memory()
        L.lbm_step_bgk_host(h_in, h_out, s, 0.7, h_taus, nsteps, h_tot, ws)
        torch.cuda.synchronize()
        assert torch.equal(h_out, want), pinned
        assert torch.equal(h_tot, want_tot), pinned
    assert L.lbm_get_status() == 0


def test_host_buffer_step_errors(lbmlib, cuda):
    import torch
    L = lbmlib
    s = L.shape(16, 8)
    h = torch.zeros(9 * 16 * 8)
    ws = torch.empty(L.lbm_host_workspace_bytes(s), dtype=torch.uint8, device=cuda)
    small = ws[: ws.numel() - 256]
    for kwargs, code in [(dict(nsteps=0, workspace=ws), "LBM_ERR_ARG"),
                         (dict(workspace=small), "LBM_ERR_WORKSPACE"),
                         (dict(workspace=None), "LBM_ERR_WORKSPACE")]:
        with pytest.raises(L.LbmError, match=code):
            L.lbm_step_bgk_host(h, None, s, 0.7, **kwargs)
    with pytest.raises(L.LbmError, match="LBM_ERR_TAU"):
        L.lbm_step_bgk_host(h, None, s, 0.5, workspace=ws)
