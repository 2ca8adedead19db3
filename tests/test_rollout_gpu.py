"""Parity of the K-step rollout training step (gnn_train_step_rollout,
through the C ABI) with the FP64 oracle's rollout loss and its reverse-mode
gradient through the dynamics (oracle.train.rollout_loss).

Stated tolerances:
  * K = 1 is the fused one-step training step: loss bitwise equal, gradient
    within 1e-5 relative L2 (the same arithmetic; the loss scale is formed
    once in double instead of float);
  * K = 2, 3 against the oracle: loss within 2e-2 relative (the loss is
    mostly the network's own corrections, whose BF16 error enters every
    step), gradient cosine
    >= 0.999 overall and per tensor >= 0.995 with relative L2 <= 5e-2 (BF16
    operands and activations in every step's forward and backward);
  * 30 AdamW steps with K = 3 lower the rollout loss.
"""
import numpy as np
import pytest

from oracle import gnn, lbm, train
from paper_2504_14494_gb300 import inputs
from gpu_util import rel_l2, to_dev

pytestmark = pytest.mark.gpu


def _cos(a, b):
    return float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300))


def _case(nb, ny, nx, K, seed, tau=0.7):
    rng = np.random.default_rng(seed)
    f0, tg = [], []
    for b in range(nb):
        f = lbm.tgv_init(nx, ny, 1.0, 0.06, 2 * np.pi / nx, 2 * np.pi / ny)
        f = f * (1 + 2e-2 * rng.standard_normal(f.shape))
        f0.append(f)
        tg.append([lbm.bgk_run(f, tau, k + 1) * (1 + 1e-3 * rng.standard_normal(f.shape))
                   for k in range(K)])
    f0 = np.stack(f0, axis=1).astype(np.float32)
    tgs = np.stack([np.stack([tg[b][k] for b in range(nb)], axis=1) for k in range(K)],
                   axis=0).astype(np.float32)                     # [K][9][nb][ny][nx]
    return f0, tgs


def _run(L, dev, theta, f0, tgs, K, tau, steps=1, lr=0.0, rollout=True):
    import torch
    nb, ny, nx = f0.shape[1:]
    s = L.shape(nx, ny, nb)
    din, _ = to_dev(f0, dev)
    dtg = torch.from_numpy(tgs.reshape(-1).copy()).to(dev)
    p = torch.from_numpy(np.asarray(theta, np.float32)).to(dev)
    pk = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=dev)
    L.gnn_pack(p, pk)
    m = torch.zeros(L.gnn_trainable_count(), device=dev)
    v = torch.zeros_like(m)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    grads = torch.zeros_like(m)
    if rollout:
        ws = torch.empty(L.gnn_rollout_workspace_bytes(s, K), dtype=torch.uint8, device=dev)
    else:
        ws = torch.empty(L.gnn_train_workspace_bytes(s), dtype=torch.uint8, device=dev)
    losses = []
    for t in range(1, steps + 1):
        if rollout:
            L.gnn_train_step_rollout(din, dtg, K, s, tau, None, p, pk, m, v, t, lr, 0.0, loss,
                                     grads, ws)
        else:
            L.gnn_train_step(din, dtg, s, tau, None, p, pk, m, v, t, lr, 0.0, loss, grads, ws)
        losses.append(loss.item())
    assert L.lbm_get_status() == 0
    return losses, grads.cpu().numpy().astype(np.float64)


def test_rollout_one_step_is_the_fused_train_step(lbmlib, cuda):
    f0, tgs = _case(2, 8, 12, 1, 3)
    theta = inputs.xavier_params(4, s_df=1e-2, bias_scale=0.1)
    (la,), ga = _run(lbmlib, cuda, theta, f0, tgs, 1, 0.7)
    (lb,), gb = _run(lbmlib, cuda, theta, f0, tgs, 1, 0.7, rollout=False)
    assert la == lb
    assert rel_l2(ga, gb) <= 1e-5


@pytest.mark.parametrize("nb,ny,nx,K,variant", [(2, 8, 12, 2, 0), (1, 9, 14, 3, 0),
                                                (2, 6, 20, 2, 2), (1, 12, 12, 3, 4)])
def test_rollout_matches_oracle(lbmlib, cuda, nb, ny, nx, K, variant):
    f0, tgs = _case(nb, ny, nx, K, 10 + nx + K)
    # s_df 1e-3 keeps three steps of a random network near the lattice's
    # own dynamics (at 1e-2 its corrections grow without bound in 3 steps)
    theta = inputs.xavier_params(20 + ny, s_df=1e-3, bias_scale=0.1, variant=variant)
    (l_gpu,), g_gpu = _run(lbmlib, cuda, theta, f0, tgs, K, 0.7)
    l_ref, g_ref = 0.0, np.zeros(gnn.N_TRAINABLE)
    for b in range(nb):
        lb, gb, _ = train.rollout_loss(f0[:, b].astype(np.float64),
                                       [tgs[k][:, b].astype(np.float64) for k in range(K)],
                                       theta, 0.7)
        l_ref += lb / nb
        g_ref += gb / nb
    assert abs(l_gpu - l_ref) <= 2e-2 * l_ref, (l_gpu, l_ref)
    assert _cos(g_gpu, g_ref) >= 0.999, _cos(g_gpu, g_ref)
    o = 0
    for name, shape in gnn.SHAPES:
        n = int(np.prod(shape))
        a, r = g_gpu[o:o + n], g_ref[o:o + n]
        o += n
        if not np.any(r):
            assert not np.any(a), name  # variant-unused tensors
            continue
        c, e = _cos(a, r), rel_l2(a, r)
        print(f"{name:12s} cos {c:.6f} relL2 {e:.2e}")
        assert c >= 0.995 and e <= 5e-2, (name, c, e)


def test_rollout_training_lowers_the_loss(lbmlib, cuda):
    f0, tgs = _case(2, 16, 16, 3, 5)
    theta = inputs.xavier_params(6, s_df=1e-4)
    losses, _ = _run(lbmlib, cuda, theta, f0, tgs, 3, 0.7, steps=30, lr=1e-3)
    print("rollout loss", losses[0], "->", losses[-1])
    assert all(np.isfinite(losses)) and losses[-1] < losses[0]

