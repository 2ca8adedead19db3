"""Pins of the FP64 GNN oracle (no GPU): special cases, brute force on tiny
lattices, library routines and finite differences."""
import numpy as np
import pytest

from oracle import gnn, lbm
from paper_2504_14494_gb300 import inputs


def _state(nx, ny, seed, u0=0.05, amp=2e-2):
    f = lbm.tgv_init(nx, ny, 1.0, u0, 2 * np.pi / nx, 2 * np.pi / ny)
    return f * inputs.perturbation(f.shape, seed, amp)


def _params(seed, bias=0.1, s_df=1e-2):
    return inputs.xavier_params(seed, s_df=s_df, bias_scale=bias)


def test_layout_matches_inputs_module():
    """The oracle's parameter layout and the shared input layout agree."""
    assert gnn.N_TRAINABLE == inputs.N_TRAINABLE == 38922
    assert gnn.N_TOTAL == inputs.N_PARAMS
    assert [s for _, s in gnn.SHAPES] == [tuple(s) for s in inputs.PARAM_SHAPES]


def test_gelu_matches_torch_tanh_gelu():
    """The GELU reading (tanh form) equals torch's gelu(approximate='tanh')
    in FP64, and its derivative equals autograd's."""
    torch = pytest.importorskip("torch")
    z = np.linspace(-8, 8, 2001)
    zt = torch.tensor(z, dtype=torch.float64, requires_grad=True)
    yt = torch.nn.functional.gelu(zt, approximate="tanh")
    yt.sum().backward()
    assert np.allclose(gnn.gelu(z), yt.detach().numpy(), rtol=1e-14, atol=1e-15)
    assert np.allclose(gnn.gelu_grad(z), zt.grad.numpy(), rtol=1e-13, atol=1e-14)


def test_bf16_round_matches_torch():
    """bfloat16 round-to-nearest-even agrees with torch's float32->bfloat16."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    a = np.concatenate([rng.standard_normal(10000).astype(np.float32),
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -1.0 - 2 ** -8, 0.0], np.float32)])
    ref = torch.tensor(a).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(gnn.bf16_round(a), ref)


@pytest.mark.parametrize("nx,ny", [(4, 4), (5, 3), (3, 3)])
def test_bruteforce_edge_mlp_equals_split_form(nx, ny):
    """W_e [h_i; h_j; e_k] = W_a h_i + W_b h_j + W_c e_k (linearity): the
    brute-force per-edge form and the split form agree to FP64 round-off."""
    p = gnn.unpack(_params(11))
    f = _state(nx, ny, 5)
    y, _ = gnn.forward(f, p)
    ys = gnn.forward_split(f, p)
    assert np.allclose(y, ys, rtol=1e-12, atol=1e-12)


def _loop_forward(f_pre, p):
    """Independent brute force with explicit coordinates and Python loops
    over nodes and the 8 neighbours (Sec. 2.2 message passing)."""
    _, ny, nx = f_pre.shape
    e = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    g = lambda z: 0.5 * z * (1.0 + np.tanh(np.sqrt(2 / np.pi) * (z + 0.044715 * z ** 3)))
    h = {}
    for y in range(ny):
        for x in range(nx):
            fi = f_pre[:, y, x]
            rho = fi.sum()
            ux = sum(fi[i] * e[i][0] for i in range(9)) / rho
            uy = sum(fi[i] * e[i][1] for i in range(9)) / rho
            xin = (np.concatenate([fi, [rho, ux, uy]]) - p["mu"]) / p["sigma"]
            h[(x, y)] = g(p["enc2.W"] @ g(p["enc1.W"] @ xin + p["enc1.b"]) + p["enc2.b"])
    for r in range(2):
        new = {}
        for (x, y), hi in h.items():
            a = np.zeros(64)
            for k in range(1, 9):
                hj = h[((x + e[k][0]) % nx, (y + e[k][1]) % ny)]
                a += g(p[f"r{r}.edge.W"] @ np.concatenate([hi, hj, e[k]]) + p[f"r{r}.edge.b"])
            new[(x, y)] = hi + g(p[f"r{r}.node.W"] @ np.concatenate([hi, a]) + p[f"r{r}.node.b"])
        h = new
    out = np.zeros((ny * nx, 10))
    for (x, y), hi in h.items():
        out[y * nx + x] = p["head.W"] @ hi + p["head.b"]
    return out


@pytest.mark.parametrize("nx,ny", [(3, 3), (4, 2)])
def test_forward_equals_loop_bruteforce(nx, ny):
    p = gnn.unpack(_params(12))
    f = _state(nx, ny, 6)
    y, _ = gnn.forward(f, p)
    assert np.allclose(y, _loop_forward(f, p), rtol=1e-12, atol=1e-12)


def test_zero_network_reduces_to_bgk():
    """Eq. 3 with all trainable values zero: y = 0, so tau_adj = 0.5 +
    sigmoid(0) = 1 and Delta f = 0, and the GNN step equals the BGK step
    (Eq. 1) exactly."""
    theta = inputs.zero_params()
    f = _state(6, 5, 8)
    a = gnn.gnn_step(f, theta, 0.7)
    b = lbm.bgk_step(f, 0.7)
    assert np.array_equal(a, b) or np.allclose(a, b, rtol=0, atol=1e-16)


def test_tau_adj_range_and_delta_f_scale():
    """Sec. 2.3.1: the sigmoid-scaled adjustment lies in (0.5, 1.5) and the
    correction is s_df times the head output."""
    p = gnn.unpack(_params(13, bias=2.0))
    y = np.random.default_rng(0).standard_normal((100, 10)) * 3
    tau_adj, df = gnn.heads(y, p)
    assert np.all(tau_adj > 0.5) and np.all(tau_adj < 1.5)
    sat, _ = gnn.heads(np.array([[-800.0] + [0] * 9, [800.0] + [0] * 9, [0.0] * 10]), p)
    assert np.allclose(sat, [0.5, 1.5, 1.0], rtol=0, atol=1e-15)
    assert np.allclose(df, p["s_df"] * y[:, 1:].T)


def test_translation_invariance():
    """The lattice graph is periodic and the network is shared over nodes:
    shifting the input field shifts the output field."""
    theta = _params(14)
    f = _state(6, 4, 9)
    a = gnn.gnn_step(f, theta, 0.9)
    b = gnn.gnn_step(np.roll(f, (1, 2), axis=(1, 2)), theta, 0.9)
    assert np.allclose(np.roll(a, (1, 2), axis=(1, 2)), b, rtol=1e-13, atol=1e-15)


def _perturbed(p, name, d, h):
    q = dict(p)
    q[name] = p[name] + h * d
    return q


def test_backward_matches_central_differences():
    """Hand-derived reverse mode vs central finite differences in FP64
    (h = 1e-6): directional derivatives along a random direction of every
    tensor, plus 40 single entries, and the gradient w.r.t. the inputs."""
    nx, ny = 4, 4
    p = gnn.unpack(_params(15, bias=0.2))
    f = _state(nx, ny, 10, u0=0.08, amp=5e-2)
    rng = np.random.default_rng(4)
    dy = rng.standard_normal((nx * ny, 10))
    J = lambda pp, ff: float(np.sum(dy * gnn.forward(ff, pp)[0]))
    _, cache = gnn.forward(f, p)
    g, df = gnn.backward(dy, cache, p)
    h = 1e-6
    for name, shape in gnn.SHAPES:
        d = rng.standard_normal(shape)
        fd = (J(_perturbed(p, name, d, h), f) - J(_perturbed(p, name, d, -h), f)) / (2 * h)
        an = float(np.sum(g[name] * d))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (name, fd, an)
    names = [n for n, _ in gnn.SHAPES]
    for _ in range(40):
        name = names[rng.integers(len(names))]
        shape = dict(gnn.SHAPES)[name]
        d = np.zeros(shape)
        idx = tuple(int(rng.integers(s)) for s in shape)
        d[idx] = 1.0
        hs = 1e-4                    # |J| ~ 1e2: keep the round-off eps|J|/h small
        fd = (J(_perturbed(p, name, d, hs), f) - J(_perturbed(p, name, d, -hs), f)) / (2 * hs)
        assert abs(fd - g[name][idx]) <= 1e-6 * max(abs(g[name][idx]), 1e-2), (name, idx)
    # inputs: relative step on the populations
    d = rng.standard_normal(f.shape) * 1e-2
    hf = 1e-5
    fd = (J(p, f + hf * d) - J(p, f - hf * d)) / (2 * hf)
    an = float(np.sum(df * d.reshape(9, -1)))
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_collide_loss_gradient_matches_central_differences():
    """Eq. 3 + Eq. 4: dL/dy from collide_loss vs central differences in y."""
    nx, ny = 4, 3
    p = gnn.unpack(_params(16, s_df=1e-3))
    f = _state(nx, ny, 11)
    target = _state(nx, ny, 12)
    rng = np.random.default_rng(5)
    y = rng.standard_normal((nx * ny, 10))
    taus = 0.6 + 0.3 * rng.random(nx * ny)
    loss, dy, _ = gnn.collide_loss(f, y, taus, target, p)
    h = 1e-6
    for _ in range(30):
        n, c = int(rng.integers(nx * ny)), int(rng.integers(10))
        yp, ym = y.copy(), y.copy()
        yp[n, c] += h
        ym[n, c] -= h
        fd = (gnn.collide_loss(f, yp, taus, target, p)[0] - gnn.collide_loss(f, ym, taus, target, p)[0]) / (2 * h)
        assert abs(fd - dy[n, c]) <= 1e-6 * abs(dy[n, c]) + 1e-14, (n, c, fd, dy[n, c])


def test_collide_loss_reduces_to_mse_of_eq3():
    """Eq. 4 is the mean over nodes x 9 of the squared difference of the Eq. 3
    output from the target; with y = 0 Eq. 3 is the BGK collision."""
    p = gnn.unpack(inputs.zero_params())
    f = _state(5, 4, 13)
    target = _state(5, 4, 14)
    loss, _, f_pred = gnn.collide_loss(f, np.zeros((20, 10)), 0.8, target, p)
    assert np.allclose(f_pred.reshape(9, 4, 5), lbm.bgk_collide(f, 0.8), rtol=0, atol=1e-16)
    assert abs(loss - np.mean((lbm.bgk_collide(f, 0.8) - target) ** 2)) < 1e-18


def test_weighted_collide_loss_gradient_and_special_cases():
    """Per-node weights in Eq. 4 (the weighted training step): the gradient
    matches central differences; all weights 1 give the plain loss; a weight
    w on one lattice scales exactly that lattice's share."""
    nx, ny = 4, 3
    p = gnn.unpack(_params(17, s_df=1e-3))
    f = _state(nx, ny, 21)
    target = _state(nx, ny, 22)
    rng = np.random.default_rng(7)
    y = rng.standard_normal((nx * ny, 10))
    w = 0.5 + rng.random(nx * ny)
    loss, dy, _ = gnn.collide_loss(f, y, 0.7, target, p, node_weight=w)
    h = 1e-6
    for _ in range(20):
        n, c = int(rng.integers(nx * ny)), int(rng.integers(10))
        yp, ym = y.copy(), y.copy()
        yp[n, c] += h
        ym[n, c] -= h
        fd = (gnn.collide_loss(f, yp, 0.7, target, p, node_weight=w)[0]
              - gnn.collide_loss(f, ym, 0.7, target, p, node_weight=w)[0]) / (2 * h)
        assert abs(fd - dy[n, c]) <= 1e-6 * abs(dy[n, c]) + 1e-14, (n, c, fd, dy[n, c])
    one = gnn.collide_loss(f, y, 0.7, target, p, node_weight=np.ones(nx * ny))
    plain = gnn.collide_loss(f, y, 0.7, target, p)
    assert one[0] == plain[0] and np.array_equal(one[1], plain[1])
    _, _, f_pred = plain
    r2 = ((f_pred - target.reshape(9, -1)) ** 2).sum(axis=0)
    w3 = np.ones(nx * ny)
    w3[:nx] = 3.0                     # the first row of nodes
    l3 = gnn.collide_loss(f, y, 0.7, target, p, node_weight=w3)[0]
    assert abs(l3 - (plain[0] + 2.0 * r2[:nx].sum() / (9 * nx * ny))) <= 1e-15


def test_pair_weights_definition():
    """D_b is the mean squared one-step BGK residual of instance b; w_b =
    mean(D) / D_b (the zero network's weighted loss then equals the plain
    one); the cap applies to an instance whose residual vanishes."""
    from oracle import train
    rng = np.random.default_rng(9)
    f_in = [_state(5, 4, 30 + b) for b in range(3)]
    taus = [0.6, 0.8, 1.1]
    tg = [lbm.bgk_step(a, t) + 1e-4 * (b + 1) * rng.standard_normal(a.shape)
          for b, (a, t) in enumerate(zip(f_in, taus))]
    tg[2] = lbm.bgk_step(f_in[2], taus[2])  # no residual at all
    d, w = train.pair_weights(f_in, tg, taus)
    for b in range(3):
        assert abs(d[b] - np.mean((lbm.bgk_step(f_in[b], taus[b]) - tg[b]) ** 2)) <= 1e-24
    assert d[2] == 0.0 and w[2] == 1.0e4
    assert np.allclose(w[:2], d.mean() / d[:2], rtol=1e-14)
    assert abs(np.mean(w[:2] * d[:2]) - d.mean()) <= 1e-15 * d.mean() * 10


# --- variants: conservative correction (2) and the MLP-only network of Fig. 2 (1) ---
def test_conservative_projection_invariants():
    """The projection removes exactly the mass and momentum of Delta f: it is
    idempotent, symmetric, and leaves already-conserving corrections alone."""
    rng = np.random.default_rng(21)
    df = rng.standard_normal((9, 40))
    P = gnn.conserve(df)
    e = lbm.E.astype(np.float64)
    assert np.allclose(P.sum(axis=0), 0.0, atol=1e-14)
    assert np.allclose(e[:, 0] @ P, 0.0, atol=1e-14)
    assert np.allclose(e[:, 1] @ P, 0.0, atol=1e-14)
    assert np.allclose(gnn.conserve(P), P, atol=1e-14)
    b = rng.standard_normal((9, 40))
    assert np.allclose(np.sum(gnn.conserve(df) * b, axis=0), np.sum(df * gnn.conserve(b), axis=0))
    # a population vector orthogonal to 1, e_x, e_y (e_x^2 - e_y^2 pattern)
    o = (e[:, 0] ** 2 - e[:, 1] ** 2)[:, None] * np.ones((1, 3))
    assert np.allclose(gnn.conserve(o), o, atol=1e-15)


def test_conservative_step_conserves_mass_and_momentum():
    """With the conservative variant the GNN step (Eq. 3) conserves mass and
    momentum exactly, like BGK; without it, Delta f moves them."""
    f = _state(6, 5, 31)
    for variant, tol in ((2, 1e-13), (0, None)):
        theta = inputs.xavier_params(33, s_df=1e-2, bias_scale=0.1, variant=variant)
        g = gnn.gnn_step(f, theta, 0.7)
        t0, t1 = lbm.totals(f), lbm.totals(g)
        drift = np.abs(t1[:3] - t0[:3]).max()
        if tol is None:
            assert drift > 1e-6
        else:
            assert drift < tol


def test_mlp_only_is_a_per_node_relu_mlp():
    """Variant 1 (Fig. 2): no message passing, so a node's output does not
    depend on its neighbours, and it equals a two-layer ReLU MLP + head
    written out per node."""
    theta = inputs.xavier_params(34, s_df=1e-2, bias_scale=0.1, variant=1)
    p = gnn.unpack(theta)
    f = _state(5, 4, 35)
    y, _ = gnn.forward(f, p)
    f2 = f.copy()
    f2[:, 0, 1] *= 1.01                      # change a neighbour of node (0, 0)
    y2, _ = gnn.forward(f2, p)
    assert np.array_equal(y[0], y2[0]) and not np.array_equal(y[1], y2[1])
    r = lambda z: np.maximum(z, 0.0)
    for n in (0, 7, 19):
        yy, xx = divmod(n, 5)
        fi = f[:, yy, xx]
        rho = fi.sum()
        u = (lbm.E.astype(np.float64).T @ fi) / rho
        xin = (np.concatenate([fi, [rho, u[0], u[1]]]) - p["mu"]) / p["sigma"]
        h = r(p["enc2.W"] @ r(p["enc1.W"] @ xin + p["enc1.b"]) + p["enc2.b"])
        assert np.allclose(y[n], p["head.W"] @ h + p["head.b"], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 6])
def test_variant_gradients_match_central_differences(variant):
    nx, ny = 4, 3
    p = gnn.unpack(inputs.xavier_params(36, s_df=1e-2, bias_scale=0.2, variant=variant))
    f = _state(nx, ny, 37, u0=0.08, amp=5e-2)
    target = _state(nx, ny, 38)
    rng = np.random.default_rng(variant)
    taus = 0.6 + 0.3 * rng.random(nx * ny)

    def loss(pp, ff):
        y, _ = gnn.forward(ff, pp)
        return gnn.collide_loss(ff, y, taus, target, pp)[0]

    y, cache = gnn.forward(f, p)
    _, dy, _ = gnn.collide_loss(f, y, taus, target, p)
    g, df = gnn.backward(dy, cache, p)
    h = 1e-5
    for name, shape in gnn.SHAPES:
        d = rng.standard_normal(shape)
        pp = dict(p); pm = dict(p)
        pp[name] = p[name] + h * d
        pm[name] = p[name] - h * d
        fd = (loss(pp, f) - loss(pm, f)) / (2 * h)
        an = float(np.sum(g[name] * d))
        assert abs(fd - an) <= 1e-5 * max(abs(an), 1e-12) + 1e-18, (variant, name, fd, an)


def test_fixed_tau_variant_ignores_the_tau_head():
    """Variant 4: tau_adj = 1 in Eq. 3 whatever the head's first row is, so
    with Delta f switched off (s_df tiny) the step is the BGK step, two
    networks differing only in that row give the same step, and the loss
    gradient of that row is zero."""
    nx, ny, tau = 5, 4, 0.65
    th = inputs.xavier_params(41, s_df=1e-2, bias_scale=0.2, variant=4)
    th2 = th.copy()
    th2[38272:38336] += 0.5           # head.W row 0
    th2[38912] -= 3.0                 # head.b[0]
    f = _state(nx, ny, 42)
    a, b = gnn.gnn_step(f, th, tau), gnn.gnn_step(f, th2, tau)
    assert np.array_equal(a, b)
    th0 = th.copy()
    th0[38336:38912] = 0.0            # head.W rows 1..9 and head.b[1..9]: Delta f = 0
    th0[38913:38922] = 0.0
    assert np.allclose(gnn.gnn_step(f, th0, tau), lbm.bgk_step(f, tau), rtol=1e-14, atol=0)
    p = gnn.unpack(th)
    fp = lbm.stream_pull(f)
    y, cache = gnn.forward(fp, p)
    _, dy, _ = gnn.collide_loss(fp, y, tau, _state(nx, ny, 43), p)
    assert not np.any(dy[:, 0])
    g, _ = gnn.backward(dy, cache, p)
    assert not np.any(g["head.W"][0]) and g["head.b"][0] == 0.0
