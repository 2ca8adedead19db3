"""Parity of the channel training path (through the C ABI) with the FP64
oracle: the forced restriction of a refined channel and the fused channel
training step (pull with bounce-back, network on the walled graph with the
forced velocity feature, Eq. 3 with Guo's source, Eq. 4, backward, AdamW).

Stated tolerances:
  * restriction: FP32 rounding of f - f^eq - P amplified by the rescale
    factor k = (1 - 1/tau_c) m tau_c / tau_f, i.e. per population
    |err| <= 1e-6 |f| + 2.4e-7 (1 + |k|) |f|;
  * training step with the zero network (tau_adj = 1, Delta f = 0 exactly):
    loss within 2e-3 relative (FP32 arithmetic on identical inputs: f*_pred
    carries ~1 ulp of f, 3e-8, against pair residuals of ~2e-5, whose
    squares average the rounding down to ~1e-4 of the loss);
  * training step with a random network: loss within 1e-2 relative (the
    network's BF16 error reaches f*_pred through Eq. 3), gradient cosine
    >= 0.999 overall and per tensor >= 0.995 with relative L2 <= 5e-2; the
    gradient of the periodic graph (walls ignored) is measurably farther.
"""
import numpy as np
import pytest

from oracle import channel, gnn, lbm, train
from paper_2504_14494_gb300 import inputs
from gpu_util import from_dev, rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _cos(a, b):
    return float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))


def _channel_state(nb, ny, nx, seed, umax=0.04):
    """Channels at rest-density with a parabolic profile and a perturbation."""
    rng = np.random.default_rng(seed)
    y = np.arange(ny)[:, None] + 0.5
    u = 4 * umax * y * (ny - y) / ny ** 2 * np.ones((1, nx))
    f = lbm.equilibrium(np.ones((ny, nx)), u, np.zeros((ny, nx)))
    f = np.stack([f * (1 + 1e-2 * rng.standard_normal(f.shape)) for _ in range(nb)], axis=1)
    return f.astype(np.float32)


@pytest.mark.parametrize("m,nb,ny,nx", [(3, 2, 5, 3), (3, 1, 32, 8), (1, 2, 4, 4), (5, 2, 3, 2),
                                        (3, 3, 7, 45)])
def test_channel_restrict_matches_oracle(lbmlib, cuda, m, nb, ny, nx):
    """lbm_restrict_channel vs the oracle's restrict_forced of the pulled fine
    state, per-lattice tau_f, tau_c and force; m = 1 is one channel BGK step."""
    import torch
    L = lbmlib
    ff = _channel_state(nb, m * ny, m * nx, seed=m + 7 * ny + nx)
    tau_c = np.array([0.55, 0.8, 1.1][:nb] + [0.7] * max(0, nb - 3), np.float32)
    tau_f = (0.5 + m * (tau_c.astype(np.float64) - 0.5)).astype(np.float32)
    gf = np.array([2e-5, 7e-5, 1e-4][:nb] + [3e-5] * max(0, nb - 3), np.float32)
    din, _ = to_dev(ff, cuda)
    out = torch.full((9 * nb * ny * nx,), float("nan"), device=cuda)
    tc_d = torch.from_numpy(tau_c).to(cuda)
    tf_d = torch.from_numpy(tau_f).to(cuda)
    g_d = torch.from_numpy(gf).to(cuda)
    L.lbm_restrict_channel(din, L.shape(m * nx, m * ny, nb), out, L.shape(nx, ny, nb), m, 0.0,
                           tf_d, 0.0, tc_d, 0.0, g_d)
    assert L.lbm_get_status() == 0
    got = from_dev(out, (9, nb, ny, nx))
    for b in range(nb):
        fb = ff[:, b].astype(np.float64)
        want = train.restrict_forced(channel.stream_pull_walls(fb), m, float(tau_f[b]),
                                     float(tau_c[b]), float(gf[b]))
        k = (1 - 1 / float(tau_c[b])) * m * float(tau_c[b]) / float(tau_f[b])
        tol = 1e-6 * np.abs(want) + 2.4e-7 * (1 + abs(k)) * np.abs(want)
        assert np.all(np.abs(got[:, b] - want) <= tol), (b, np.abs(got[:, b] - want).max())
        if m == 1:
            step = channel.channel_step(fb, float(tau_c[b]), float(gf[b]))
            assert np.allclose(got[:, b], step, rtol=2e-6, atol=0)
    # scalar force and times give the same as the arrays filled with them
    out2 = torch.empty_like(out)
    L.lbm_restrict_channel(din, L.shape(m * nx, m * ny, nb), out2, L.shape(nx, ny, nb), m,
                           float(tau_f[0]), None, float(tau_c[0]), None, float(gf[0]))
    out3 = torch.empty_like(out)
    L.lbm_restrict_channel(din, L.shape(m * nx, m * ny, nb), out3, L.shape(nx, ny, nb), m, 0.0,
                           torch.full((nb,), float(tau_f[0]), device=cuda), 0.0,
                           torch.full((nb,), float(tau_c[0]), device=cuda), 0.0,
                           torch.full((nb,), float(gf[0]), device=cuda))
    assert torch.equal(out2, out3)


def _pairs(ny, nx, taus, umax, n_steps):
    """Oracle channel pairs (refined 3x, restricted), one lattice per tau."""
    f_in, f_tg, g = [], [], []
    for t in taus:
        gc = 8 * lbm.viscosity(t) * umax / ny ** 2
        a, b = train.channel_pair(ny, nx, t, gc, n_steps)
        f_in.append(a)
        f_tg.append(b)
        g.append(gc)
    return (np.stack(f_in, axis=1).astype(np.float32), np.stack(f_tg, axis=1).astype(np.float32),
            np.array(g, np.float32))


def _oracle_step(theta, f_in, f_tg, taus, gs, walls=True):
    """Loss and gradient of the oracle's channel training step on a stack."""
    pr = gnn.unpack(theta)
    nb = f_in.shape[1]
    ny, nx = f_in.shape[2], f_in.shape[3]
    per = ny * nx
    fpre = [channel.stream_pull_walls(f_in[:, b].astype(np.float64)) for b in range(nb)]
    outs = [gnn.forward(fpre[b], pr, walls=walls, force_x=float(gs[b])) for b in range(nb)]
    y = np.concatenate([o[0] for o in outs], axis=0)
    stack = np.concatenate(fpre, axis=1)               # (9, nb*ny, nx), b-major nodes
    tgt = np.concatenate([f_tg[:, b].astype(np.float64) for b in range(nb)], axis=1)
    tau_n = np.repeat(np.asarray(taus, np.float32).astype(np.float64), per)
    g_n = np.repeat(np.asarray(gs, np.float64), per)
    loss, dy, _ = channel.collide_loss_channel(stack, y, tau_n, tgt, pr, g_n)
    g_ref = np.zeros(gnn.N_TRAINABLE)
    for b in range(nb):
        g, _ = gnn.backward(dy[b * per:(b + 1) * per], outs[b][1], pr)
        g_ref += gnn.pack_grads(g)
    return loss, g_ref


def _gpu_step(L, dev, theta, f_in, f_tg, taus, gs, lr=0.0, steps=1, scalar=False):
    import torch
    nb, ny, nx = f_in.shape[1:]
    s = L.shape(nx, ny, nb)
    din, _ = to_dev(f_in, dev)
    dtg, _ = to_dev(f_tg, dev)
    p = torch.from_numpy(np.asarray(theta, np.float32)).to(dev)
    pk = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=dev)
    L.gnn_pack(p, pk)
    m = torch.zeros(L.gnn_trainable_count(), device=dev)
    v = torch.zeros_like(m)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    grads = torch.zeros_like(m)
    ws = torch.empty(L.gnn_train_workspace_bytes(s), dtype=torch.uint8, device=dev)
    td = torch.from_numpy(np.asarray(taus, np.float32)).to(dev)
    gd = torch.from_numpy(np.asarray(gs, np.float32)).to(dev)
    losses = []
    for t in range(1, steps + 1):
        if scalar:
            L.gnn_train_step_channel(din, dtg, s, float(taus[0]), None, float(gs[0]), None, None,
                                     p, pk, m, v, t, lr, 0.0, loss, grads, ws)
        else:
            L.gnn_train_step_channel(din, dtg, s, 0.0, td, 0.0, gd, None, p, pk, m, v, t, lr, 0.0,
                                     loss, grads, ws)
        losses.append(loss.item())
    assert L.lbm_get_status() == 0
    return losses, grads.cpu().numpy().astype(np.float64)


def test_channel_train_step_zero_network_loss_is_exact(lbmlib, cuda):
    """All-zero network: the prediction is one BGK channel step with Guo's
    source, so the GPU loss equals the oracle's to FP32 rounding."""
    f_in, f_tg, gs = _pairs(8, 6, [0.6, 0.9], 0.04, 12)
    theta = inputs.zero_params()
    (l_gpu,), g_gpu = _gpu_step(lbmlib, cuda, theta, f_in, f_tg, [0.6, 0.9], gs)
    l_ref, g_ref = _oracle_step(theta, f_in, f_tg, [0.6, 0.9], gs)
    assert abs(l_gpu - l_ref) <= 2e-3 * l_ref, (l_gpu, l_ref)
    assert _cos(g_gpu, g_ref) >= 0.999


@pytest.mark.parametrize("nb,ny,nx,scalar", [(3, 12, 10, False), (2, 4, 40, False),
                                             (1, 9, 14, True)])
def test_channel_train_step_matches_oracle(lbmlib, cuda, nb, ny, nx, scalar):
    """One fused channel training step with a random network: loss and
    gradient against the oracle on the walled graph, and farther from the
    oracle's gradient on the periodic graph."""
    taus = [0.6, 0.75, 0.95][:nb] if not scalar else [0.7]
    f_in, f_tg, gs = _pairs(ny, nx, taus, 0.04, 10)
    theta = inputs.xavier_params(40 + ny, s_df=1e-3, bias_scale=0.1)
    (l_gpu,), g_gpu = _gpu_step(lbmlib, cuda, theta, f_in, f_tg, taus, gs, scalar=scalar)
    l_ref, g_ref = _oracle_step(theta, f_in, f_tg, taus, gs)
    assert abs(l_gpu - l_ref) <= 1e-2 * l_ref, (l_gpu, l_ref)
    assert _cos(g_gpu, g_ref) >= 0.999, _cos(g_gpu, g_ref)
    o = 0
    for name, shape in gnn.SHAPES:
        n = int(np.prod(shape))
        a, r = g_gpu[o:o + n], g_ref[o:o + n]
        o += n
        c, e = _cos(a, r), rel_l2(a, r)
        print(f"{name:12s} cos {c:.6f} relL2 {e:.2e}")
        assert c >= 0.995 and e <= 5e-2, (name, c, e)
    _, g_per = _oracle_step(theta, f_in, f_tg, taus, gs, walls=False)
    assert rel_l2(g_gpu, g_ref) < 0.5 * rel_l2(g_gpu, g_per)


def test_channel_training_lowers_the_loss(lbmlib, cuda):
    """30 AdamW steps on a fixed batch of restricted channel pairs lower the
    loss of the channel network."""
    taus = [0.6, 0.8]
    f_in, f_tg, gs = _pairs(10, 4, taus, 0.04, 15)
    theta = inputs.xavier_params(5, s_df=1e-4)
    losses, _ = _gpu_step(lbmlib, cuda, theta, f_in, f_tg, taus, gs, lr=1e-3, steps=30)
    print("loss", losses[0], "->", losses[-1])
    assert all(np.isfinite(losses))
    assert losses[-1] < losses[0]


def test_channel_pair_bank_matches_oracle_pairs(lbmlib, cuda):
    """A small ChannelPairBank: every (group, snapshot) block holds the
    oracle's channel_pair of each of its lattices (refined 3x from rest,
    restricted before and after m fine steps), with its tau and coarse
    force; the blocks' order is a permutation and batch views address them."""
    from paper_2504_14494_gb300.train import ChannelPairBank
    h, nx, per = 6, 2, 2
    bank = ChannelPairBank(cuda, h=h, nx=nx, groups=2, per_group=per, snapshots=(0.1, 0.5, 1.0),
                           seed=3, u_range=(0.03, 0.05), re_range=(5.0, 20.0))
    assert lbmlib.lbm_get_status() == 0
    assert bank.nb == 2 * 3 * per
    f_in = from_dev(bank.f_in, (9, bank.nb, h, nx))
    f_tg = from_dev(bank.f_tg, (9, bank.nb, h, nx))
    tau_c = bank.tau_c.cpu().numpy()
    force = bank.force.cpu().numpy()
    seen = set()
    for grp in bank.groups:
        for t in grp["times"]:
            # find the block of this group and time: lattices with the group's taus
            for i, tc in enumerate(grp["tau_c"]):
                a, b = train.channel_pair(h, nx, float(np.float32(tc)), float(np.float32(grp["force"])),
                                          t)
                hits = [j for j in range(bank.nb)
                        if abs(tau_c[j] - tc) < 1e-7 and abs(force[j] - np.float32(grp["force"])) < 1e-12
                        and np.allclose(f_in[:, j], a, rtol=5e-5, atol=0)]
                assert len(hits) == 1, (grp["times"], t, i, len(hits))
                j = hits[0]
                assert np.allclose(f_tg[:, j], b, rtol=5e-5, atol=0)
                seen.add(j)
    assert seen == set(range(bank.nb))
    fi, ft, s, taus, forces = bank.batch_view(1, 4)
    assert (s.nx, s.ny, s.nb, s.plane_stride) == (nx, h, 4, bank.nb * h * nx)
    assert fi.data_ptr() == bank.f_in.data_ptr() + 4 * h * nx * 4
    assert np.array_equal(taus.cpu().numpy(), tau_c[4:8])


def test_channel_relative_weights_match_oracle_residuals(lbmlib, cuda):
    """The channel trainer's per-lattice residuals D_b (the zero network's
    loss on each lattice alone) equal the oracle's mean squared one-step
    residual of the BGK channel step, and its relative weights are
    mean(D) / D_b."""
    from paper_2504_14494_gb300.train import ChannelPairBank, ChannelTrainer
    h, nx = 6, 2
    bank = ChannelPairBank(cuda, h=h, nx=nx, groups=2, per_group=2, snapshots=(0.1, 1.0), seed=4,
                           u_range=(0.03, 0.05), re_range=(5.0, 20.0))
    tr = ChannelTrainer(cuda, bank, theta=inputs.xavier_params(0, s_df=1e-3), batch=4,
                        weighting="relative")
    assert lbmlib.lbm_get_status() == 0
    f_in = from_dev(bank.f_in, (9, bank.nb, h, nx))
    f_tg = from_dev(bank.f_tg, (9, bank.nb, h, nx))
    tau_c = bank.tau_c.cpu().numpy().astype(np.float64)
    force = bank.force.cpu().numpy().astype(np.float64)
    d_ref = np.array([np.mean((channel.channel_step(f_in[:, j], tau_c[j], force[j])
                               - f_tg[:, j]) ** 2) for j in range(bank.nb)])
    d_gpu = tr.lattice_residuals(bank)
    assert np.allclose(d_gpu, d_ref, rtol=5e-3, atol=0), (d_gpu, d_ref)
    w = tr.lat_w.cpu().numpy()
    assert np.allclose(w, d_gpu.mean() / d_gpu, rtol=1e-6)
    tr.step()
    assert np.isfinite(tr.loss.item()) and lbmlib.lbm_get_status() == 0
