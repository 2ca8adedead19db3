"""Pins of the FP64 channel (Poiseuille) oracle (no GPU): exact mass
conservation with walls and force, the steady profile's exact curvature
-G/nu (Eq. 5's second derivative), symmetry, and second-order convergence of
the velocity error (Eq. 6) because the wall slip is a fixed multiple of
G/nu."""
import numpy as np

from oracle import channel, lbm


def _rest(ny, nx):
    return lbm.equilibrium(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))


def _steady(ny, tau, g, nx=1):
    nu = lbm.viscosity(tau)
    steps = int(35 * ny * ny / (np.pi ** 2 * nu)) + 50
    return channel.channel_run(_rest(ny, nx), tau, g, steps)


def test_channel_conserves_mass_and_source_carries_force():
    """Bounce-back walls conserve mass; the Guo source adds no mass and adds
    exactly the force (1 - 1/(2 tau)) G per node... together with the F/2
    velocity shift the momentum gain per step and node is G minus the wall
    friction, so mass is conserved to round-off."""
    f = _rest(6, 5) * (1 + 1e-3 * np.random.default_rng(0).standard_normal((9, 6, 5)))
    m0 = f.sum()
    g = channel.channel_run(f, 0.8, 1e-5, 500)
    assert abs(g.sum() - m0) / m0 < 1e-13
    s = channel.guo_source(np.full(4, 0.03), np.full(4, -0.01), 0.8, 1e-4)
    assert np.allclose(s.sum(axis=0), 0.0, atol=1e-20)
    ex = lbm.E[:, 0].astype(np.float64)
    assert np.allclose(ex @ s, (1 - 0.5 / 0.8) * 1e-4, rtol=1e-12)


def test_steady_profile_has_exact_curvature_and_symmetry():
    ny, tau, g = 8, 1.0, 1e-6
    f = _steady(ny, tau, g)
    _, ux, uy = channel.moments_forced(f, g)
    u = ux[:, 0]
    nu = lbm.viscosity(tau)
    d2 = u[2:] - 2 * u[1:-1] + u[:-2]
    assert np.allclose(d2, -g / nu, rtol=1e-9, atol=0)
    assert np.allclose(u, u[::-1], rtol=1e-12)
    assert np.abs(uy).max() < 1e-14          # round-off of O(1) populations
    # the offset from Eq. 5 is a constant wall slip
    slip = u - channel.poiseuille_profile(ny, tau, g)
    assert np.ptp(slip) < 1e-9 * u.max()


def test_velocity_error_converges_at_second_order():
    """Eq. 6: H = 8, 16, 32 at fixed tau and fixed centre-line velocity
    (G = 8 nu u_max / H^2): max error / u_max falls as H^-2."""
    tau, umax = 1.0, 0.01
    nu = lbm.viscosity(tau)
    errs = []
    hs = [8, 16, 32]
    for h in hs:
        g = 8 * nu * umax / h ** 2
        _, ux, _ = channel.moments_forced(_steady(h, tau, g), g)
        errs.append(np.abs(ux[:, 0] - channel.poiseuille_profile(h, tau, g)).max() / umax)
    for i in range(2):
        alpha = lbm.convergence_rate(errs[i], errs[i + 1], 1.0 / hs[i], 1.0 / hs[i + 1])
        assert abs(alpha - 2.0) < 0.01, (alpha, errs)


def _net(seed, variant=0, s_df=1e-2):
    from paper_2504_14494_gb300 import inputs
    return inputs.xavier_params(seed, s_df=s_df, bias_scale=0.1, variant=variant)


def test_gnn_channel_step_with_zero_network_is_the_bgk_channel_step():
    """All trainable values zero: tau_adj = 1, Delta f = 0, so the GNN channel
    step (Eq. 3 with Guo forcing) is the BGK channel step exactly."""
    from paper_2504_14494_gb300 import inputs
    f = _rest(6, 5) * (1 + 1e-2 * np.random.default_rng(1).standard_normal((9, 6, 5)))
    a = channel.gnn_channel_step(f, inputs.zero_params(), 0.7, 2e-5)
    b = channel.channel_step(f, 0.7, 2e-5)
    assert np.allclose(a, b, rtol=1e-15, atol=1e-17)


def test_gnn_channel_messages_stop_at_the_walls():
    """Brute force on a 3 x 4 channel: a node's aggregated message sums GELU
    of the edge MLP over the neighbours inside the channel only (periodic in
    x); the first and last rows have 5 neighbours, the middle rows 8."""
    from oracle import gnn
    nx, ny = 3, 4
    p = gnn.unpack(_net(3))
    f = lbm.equilibrium(np.ones((ny, nx)), np.full((ny, nx), 0.02), np.zeros((ny, nx)))
    f = f * (1 + 1e-2 * np.random.default_rng(4).standard_normal(f.shape))
    _, cache = gnn.forward(f, p, walls=True, force_x=1e-4)
    h0 = cache["h"][0]
    We, be = p["r0.edge.W"], p["r0.edge.b"]
    for y in range(ny):
        for x in range(nx):
            a, cnt = np.zeros(64), 0
            for k in range(1, 9):
                yy = y + lbm.E[k, 1]
                if yy < 0 or yy >= ny:
                    continue
                j = yy * nx + (x + lbm.E[k, 0]) % nx
                inp = np.concatenate([h0[y * nx + x], h0[j], lbm.E[k].astype(float)])
                a += gnn.gelu(We @ inp + be)
                cnt += 1
            assert cnt == (5 if y in (0, ny - 1) else 8)
            assert np.allclose(cache["a"][0][y * nx + x], a, rtol=1e-13, atol=1e-15)


def test_gnn_channel_features_use_the_forced_velocity():
    """The velocity feature is (sum f e + F/2) / rho."""
    from oracle import gnn
    p = gnn.unpack(_net(5))
    f = _rest(4, 3) * (1 + 1e-2 * np.random.default_rng(6).standard_normal((9, 4, 3)))
    _, raw = gnn.features(f, p, force_x=3e-3)
    rho, ux, uy = channel.moments_forced(f, 3e-3)
    assert np.allclose(raw[:, 10], ux.ravel(), rtol=1e-15, atol=0)
    assert np.allclose(raw[:, 11], uy.ravel(), rtol=1e-15, atol=0)


def test_gnn_channel_step_commutes_with_x_shifts():
    """The channel is periodic in x: shifting the state in x commutes with
    the GNN channel step."""
    f = _rest(5, 6) * (1 + 1e-2 * np.random.default_rng(8).standard_normal((9, 5, 6)))
    th = _net(7)
    a = np.roll(channel.gnn_channel_step(f, th, 0.75, 1e-4), 2, axis=2)
    b = channel.gnn_channel_step(np.roll(f, 2, axis=2), th, 0.75, 1e-4)
    assert np.allclose(a, b, rtol=1e-13, atol=1e-16)


def test_walled_backward_matches_central_differences():
    """Reverse mode on the channel's graph with a body force (edges across
    the walls left out, forced velocity feature) vs central differences in
    FP64: directional derivatives of every tensor and of the inputs."""
    from oracle import gnn
    nx, ny = 3, 4
    p = gnn.unpack(_net(21, s_df=1e-2))
    rng = np.random.default_rng(22)
    f = lbm.equilibrium(np.ones((ny, nx)), np.full((ny, nx), 0.03), np.zeros((ny, nx)))
    f = f * (1 + 3e-2 * rng.standard_normal(f.shape))
    gx = 2e-3
    dy = rng.standard_normal((nx * ny, 10))
    J = lambda pp, ff: float(np.sum(dy * gnn.forward(ff, pp, walls=True, force_x=gx)[0]))
    _, cache = gnn.forward(f, p, walls=True, force_x=gx)
    g, df = gnn.backward(dy, cache, p)
    h = 1e-6
    for name, shape in gnn.SHAPES:
        d = rng.standard_normal(shape)
        q1, q2 = dict(p), dict(p)
        q1[name] = p[name] + h * d
        q2[name] = p[name] - h * d
        fd = (J(q1, f) - J(q2, f)) / (2 * h)
        an = float(np.sum(g[name] * d))
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3), (name, fd, an)
    d = rng.standard_normal(f.shape) * 1e-2
    hf = 1e-5
    fd = (J(p, f + hf * d) - J(p, f - hf * d)) / (2 * hf)
    an = float(np.sum(df * d.reshape(9, -1)))
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)
    # the periodic graph's gradient differs: the mask is in effect
    _, cache_p = gnn.forward(f, p, walls=False, force_x=gx)
    gp, _ = gnn.backward(dy, cache_p, p)
    assert np.abs(gp["r0.edge.W"] - g["r0.edge.W"]).max() > 1e-3 * np.abs(g["r0.edge.W"]).max()


def test_channel_loss_gradient_matches_central_differences():
    """The channel loss (Eq. 3 with Guo's source at tau tau_adj, Eq. 4):
    dL/dy vs central differences, per-node tau and force."""
    from oracle import gnn
    nx, ny = 4, 3
    p = gnn.unpack(_net(23, s_df=1e-3))
    rng = np.random.default_rng(24)
    f = _rest(ny, nx) * (1 + 2e-2 * rng.standard_normal((9, ny, nx)))
    target = _rest(ny, nx) * (1 + 2e-2 * rng.standard_normal((9, ny, nx)))
    y = rng.standard_normal((nx * ny, 10))
    taus = 0.55 + 0.4 * rng.random(nx * ny)
    gx = 1e-3 * (1 + rng.random(nx * ny))
    loss, dy, _ = channel.collide_loss_channel(f, y, taus, target, p, gx)
    L = lambda yy: channel.collide_loss_channel(f, yy, taus, target, p, gx)[0]
    h = 1e-6
    for _ in range(30):
        n, c = int(rng.integers(nx * ny)), int(rng.integers(10))
        yp, ym = y.copy(), y.copy()
        yp[n, c] += h
        ym[n, c] -= h
        fd = (L(yp) - L(ym)) / (2 * h)
        assert abs(fd - dy[n, c]) <= 1e-6 * abs(dy[n, c]) + 1e-14, (n, c, fd, dy[n, c])


def test_channel_loss_special_cases():
    """Zero network: the prediction is the BGK channel collision, so on the
    pulled state it equals one channel step; without force the loss is the
    periodic one (Eq. 3 + Eq. 4)."""
    from oracle import gnn
    from paper_2504_14494_gb300 import inputs
    rng = np.random.default_rng(25)
    fpost = _rest(5, 4) * (1 + 1e-2 * rng.standard_normal((9, 5, 4)))
    target = _rest(5, 4) * (1 + 1e-2 * rng.standard_normal((9, 5, 4)))
    p0 = gnn.unpack(inputs.zero_params())
    fpre = channel.stream_pull_walls(fpost)
    loss, dy, pred = channel.collide_loss_channel(fpre, np.zeros((20, 10)), 0.8, target, p0, 3e-4)
    step = channel.channel_step(fpost, 0.8, 3e-4)
    assert np.allclose(pred.reshape(9, 5, 4), step, rtol=0, atol=1e-16)
    assert abs(loss - np.mean((step - target) ** 2)) < 1e-18
    p = gnn.unpack(_net(26, s_df=1e-3))
    y = rng.standard_normal((20, 10))
    a = channel.collide_loss_channel(fpre, y, 0.7, target, p, 0.0)
    b = gnn.collide_loss(fpre, y, 0.7, target, p)
    assert abs(a[0] - b[0]) <= 1e-15 * b[0]
    assert np.allclose(a[1], b[1], rtol=1e-13, atol=1e-20)


# ---- the channel's rollout loss (adjoints with walls and force) ----------------------
def test_walled_stream_adjoint_is_the_transpose():
    """<stream_pull_walls(f), g> = <f, stream_pull_walls_adjoint(g)>."""
    rng = np.random.default_rng(71)
    for ny, nx in ((1, 3), (4, 5), (6, 2)):
        f = rng.standard_normal((9, ny, nx))
        g = rng.standard_normal((9, ny, nx))
        a = float(np.sum(channel.stream_pull_walls(f) * g))
        b = float(np.sum(f * channel.stream_pull_walls_adjoint(g)))
        assert abs(a - b) <= 1e-12 * max(abs(a), 1.0), (ny, nx, a, b)


def _gnn_channel_collide(fpre, y, tau, p, gx):
    from oracle import gnn
    q, ny, nx = fpre.shape
    tau_adj, dfc = gnn.heads(y, p)
    teff = (tau * tau_adj).reshape(ny, nx)
    rho, ux, uy = channel.moments_forced(fpre, gx)
    feq = lbm.equilibrium(rho, ux, uy)
    return fpre - (fpre - feq) / teff + channel.guo_source(ux, uy, teff, gx) + dfc.reshape(q, ny, nx)


def test_channel_collide_adjoint_matches_central_differences():
    """The explicit part of the channel collision's reverse mode (y held
    fixed; f^eq and Guo's source through the forced velocity) and dL/dy
    against central differences, variants 0, 2 and 4."""
    from oracle import gnn
    for variant in (0, 2, 4):
        rng = np.random.default_rng(72 + variant)
        f = _rest(3, 4) * (1 + 2e-2 * rng.standard_normal((9, 3, 4)))
        p = gnn.unpack(_net(8, variant=variant))
        y = rng.standard_normal((12, 10))
        g = rng.standard_normal((9, 12))
        gx = 3e-3
        dy, df = channel.collide_adjoint_channel(f, y, 0.8, p, gx, g)
        J = lambda ff, yy: float(np.sum(g * _gnn_channel_collide(ff, yy, 0.8, p, gx).reshape(9, -1)))
        d = rng.standard_normal(f.shape)
        h = 1e-6
        fd = (J(f + h * d, y) - J(f - h * d, y)) / (2 * h)
        assert abs(fd - float(np.sum(df * d.reshape(9, -1)))) <= 1e-7 * abs(fd), variant
        dd = rng.standard_normal(y.shape)
        fd = (J(f, y + h * dd) - J(f, y - h * dd)) / (2 * h)
        an = float(np.sum(dy * dd))
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-12), variant


def test_channel_rollout_one_step_is_the_channel_loss():
    """K = 1: the channel rollout loss and gradient are the channel loss
    (Eq. 3 with Guo's source, Eq. 4) with the walled network's backward."""
    from oracle import gnn
    rng = np.random.default_rng(73)
    f0 = _rest(5, 4) * (1 + 1e-2 * rng.standard_normal((9, 5, 4)))
    tg = channel.channel_step(f0, 0.7, 2e-4) * (1 + 1e-3 * rng.standard_normal((9, 5, 4)))
    theta = _net(9, s_df=1e-2)
    loss, grads, _ = channel.rollout_loss_channel(f0, [tg], theta, 0.7, 2e-4)
    p = gnn.unpack(theta)
    fpre = channel.stream_pull_walls(f0)
    y, cache = gnn.forward(fpre, p, walls=True, force_x=2e-4)
    l1, dy, _ = channel.collide_loss_channel(fpre, y, 0.7, tg, p, 2e-4)
    g1 = gnn.pack_grads(gnn.backward(dy, cache, p)[0])
    assert abs(loss - l1) <= 1e-13 * l1
    assert np.allclose(grads, g1, rtol=1e-9, atol=1e-18)


def test_channel_rollout_gradient_matches_central_differences():
    """K = 2 on a walled, forced 4 x 3 channel: the reverse-mode gradient
    w.r.t. every parameter tensor and the initial state against central
    differences of the loss in FP64."""
    from oracle import gnn
    rng = np.random.default_rng(74)
    f0 = _rest(4, 3) * (1 + 2e-2 * rng.standard_normal((9, 4, 3)))
    gx = 5e-4
    tgs = [channel.channel_run(f0, 0.75, gx, k + 1) * (1 + 1e-3 * rng.standard_normal((9, 4, 3)))
           for k in range(2)]
    p = gnn.unpack(_net(10, s_df=1e-2))
    loss, grads, df0 = channel.rollout_loss_channel(f0, tgs, p, 0.75, gx)
    L = lambda pp, ff: channel.rollout_loss_channel(ff, tgs, pp, 0.75, gx)[0]
    h = 1e-6
    o = 0
    for name, shape in gnn.SHAPES:
        n = int(np.prod(shape))
        d = rng.standard_normal(shape)
        an = float(np.dot(grads[o:o + n], d.ravel()))
        o += n
        q1, q2 = dict(p), dict(p)
        q1[name] = p[name] + h * d
        q2[name] = p[name] - h * d
        fd = (L(q1, f0) - L(q2, f0)) / (2 * h)
        assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-3 * loss), (name, fd, an)
    d = rng.standard_normal(f0.shape) * 1e-2
    fd = (L(p, f0 + 1e-4 * d) - L(p, f0 - 1e-4 * d)) / 2e-4
    an = float(np.sum(df0 * d))
    assert abs(fd - an) <= 2e-5 * abs(an), (fd, an)
