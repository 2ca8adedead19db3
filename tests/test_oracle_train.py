"""Pins of the training-side oracle (no GPU): restriction special cases,
AdamW against torch's implementation and its first-step closed form."""
import numpy as np
import pytest

from oracle import lbm, train
from paper_2504_14494_gb300 import inputs


def test_fine_tau_keeps_physical_viscosity():
    """Acoustic scaling (dx, dt both / m): nu_f = m nu_c in lattice units."""
    for tau_c in (0.51, 0.8, 1.7):
        for m in (1, 2, 4):
            assert abs(lbm.viscosity(train.fine_tau(tau_c, m)) - m * lbm.viscosity(tau_c)) < 1e-15


def test_restrict_factor_one_is_identity():
    """m = 1 with tau_f = tau_c: the restriction returns its input."""
    f = lbm.tgv_init(6, 5, 1.0, 0.05, 1.0, 1.2) * inputs.perturbation((9, 5, 6), 1, 1e-2)
    assert np.allclose(train.restrict(f, 1, 0.8, 0.8), f, rtol=0, atol=1e-15)


def test_restrict_uniform_flow_is_coarse_equilibrium():
    """A uniform-flow equilibrium has no non-equilibrium part: it restricts
    to the coarse equilibrium of the same rho, u exactly."""
    rho = np.full((8, 8), 1.02)
    ux = np.full((8, 8), 0.03)
    uy = np.full((8, 8), -0.01)
    fine = lbm.equilibrium(rho, ux, uy)
    out = train.restrict(fine, 4, train.fine_tau(0.7, 4), 0.7)
    assert out.shape == (9, 2, 2)
    assert np.allclose(out, lbm.equilibrium(rho[::4, ::4], ux[::4, ::4], uy[::4, ::4]), rtol=0, atol=1e-16)


def test_restrict_injects_moments():
    """rho and u of the restricted state equal the fine node's (collision and
    the non-equilibrium rescale conserve them)."""
    f = lbm.tgv_init(16, 16, 1.0, 0.05, 2 * np.pi / 16, 2 * np.pi / 16)
    f = lbm.bgk_run(f * inputs.perturbation(f.shape, 2, 1e-3), 0.9, 3)
    c = train.restrict(f, 4, 0.9, 0.6)
    a = lbm.moments(f[:, ::4, ::4])
    b = lbm.moments(c)
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-13, atol=1e-14)


def test_restricted_pair_is_close_to_one_coarse_bgk_step():
    """The restricted fine solution is a consistent coarse state: one coarse
    BGK step from the restricted state at n lands near the restricted state
    at n+1 -- over 10x closer than with the non-equilibrium part rescaled by
    1, m or 1/m instead of m tau_c/tau_f (which pins the rescale's direction
    and size)."""
    n_c, m, u0, tau_c = 16, 4, 0.05, 0.6
    tau_f = train.fine_tau(tau_c, m)
    f_in, f_tg = train.tgv_pair(n_c, u0, 1, tau_c, 3, m)
    err = np.abs(lbm.bgk_step(f_in, tau_c) - f_tg).max()
    assert err < 1e-4
    n_f = m * n_c
    k_f = 2 * np.pi / n_f
    f = lbm.bgk_run(lbm.tgv_init(n_f, n_f, 1.0, u0, k_f, k_f), tau_f, 3 * m)
    g = lbm.bgk_run(f, tau_f, m)

    def restrict_with(ff, fac):
        sub = ff[:, ::m, ::m]
        feq = lbm.equilibrium(*lbm.moments(sub))
        return feq + (1 - 1 / tau_c) * fac * (sub - feq) / (1 - 1 / tau_f)

    assert np.allclose(restrict_with(f, m * tau_c / tau_f), f_in, rtol=0, atol=1e-15)
    for fac in (1.0, float(m), 1.0 / m):
        wrong = np.abs(lbm.bgk_step(restrict_with(f, fac), tau_c) - restrict_with(g, fac)).max()
        assert err < 0.1 * wrong, (fac, err, wrong)


def test_adamw_matches_torch():
    """The AdamW reading equals torch.optim.AdamW (decoupled weight decay) over
    5 steps."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    theta0 = rng.standard_normal(50)
    grads = [rng.standard_normal(50) for _ in range(5)]
    pt = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.AdamW([pt], lr=1e-3, betas=(0.9, 0.999), eps=1e-8, weight_decay=1e-2)
    th, m, v = theta0.copy(), np.zeros(50), np.zeros(50)
    for t, g in enumerate(grads, start=1):
        pt.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        th, m, v = train.adamw_step(th, g, m, v, t, 1e-3, 1e-2)
    assert np.allclose(th, pt.detach().numpy(), rtol=1e-14, atol=1e-15)


def test_adamw_first_step_closed_form():
    """At t = 1 the bias corrections give mhat = g, vhat = g^2, so the update
    is theta (1 - lr wd) - lr g / (|g| + eps)."""
    g = np.array([1e-3, -2.0, 0.0, 5e-9])
    th = np.array([1.0, -1.0, 0.5, 2.0])
    out, _, _ = train.adamw_step(th, g, np.zeros(4), np.zeros(4), 1, 1e-2, 0.1)
    assert np.allclose(out, th * (1 - 1e-3) - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-14, atol=1e-16)


# ---- the forced (channel) restriction ---------------------------------------------
def _accelerating(tau, g, n, shape=(3, 3), u0=0.02, v0=0.01):
    """A uniform flow under a uniform force, n LBM steps with Guo's scheme
    (streaming is the identity on a uniform state).  Starts at time-level
    velocity (u0, v0): the stored post-collision state carries j = rho u + F/2."""
    from oracle import channel
    f = lbm.equilibrium(np.ones(shape), np.full(shape, u0 + g / 2), np.full(shape, v0))
    for _ in range(n):
        rho, ux, uy = channel.moments_forced(f, g)
        f = f - (f - lbm.equilibrium(rho, ux, uy)) / tau + channel.guo_source(ux, uy, tau, g)
    return f


@pytest.mark.parametrize("tau_c", [0.55, 0.6, 0.9, 1.3])
def test_restrict_forced_accelerating_flow_is_the_coarse_state(tau_c):
    """A uniformly accelerated flow is the same physical flow on both
    lattices: the fine pre-collision state after 3n steps (F/3, tau_f)
    restricts to the coarse lattice's own state after n steps (F, tau_c) to
    round-off, although its non-equilibrium part is all force and time
    derivative; the force part taken as gradient part, dropped, scaled by m
    or the gradient scale without its m all miss by over 10 %."""
    from oracle import channel
    m, gc, nc = 3, 2e-4, 60
    tf, gf = train.fine_tau(tau_c, m), gc / m
    fc = _accelerating(tau_c, gc, nc)
    fpre = _accelerating(tf, gf, m * nc - 1)   # = the pull of the stored state
    r = train.restrict_forced(fpre, m, tf, tau_c, gf)
    rho, jx, uy = lbm.moments(fc)
    scale = np.abs(fc - lbm.equilibrium(rho, jx - gc / 2 / rho, uy)).max()
    assert np.abs(r - fc).max() < 1e-7 * scale
    sub = fpre[:, 1::3, 1::3]
    rr, a, b = channel.moments_forced(sub, gf)
    fe = lbm.equilibrium(rr, a, b)
    pf = (tf - 0.5) * channel.guo_term(a, b, gf)
    k = (1 - 1 / tau_c) * m * tau_c / tf
    for wrong in (fe + k * (sub - fe), fe + k * (sub - fe - pf),
                  fe + k * (sub - fe - pf) + m * pf,
                  fe + (k / m) * (sub - fe - pf) + pf):
        assert np.abs(wrong - fc).max() > 0.1 * scale


def test_restrict_forced_without_force_is_the_post_collision_restriction():
    """F = 0: restricting the pre-collision state equals restricting the
    post-collision state that one BGK collision makes of it (the periodic
    reading), with the fine node (3I + 1, 3J + 1) as the co-located one."""
    rng = np.random.default_rng(31)
    fpre = lbm.tgv_init(9, 12, 1.0, 0.04, 2 * np.pi / 9, 2 * np.pi / 12)
    fpre = fpre * (1 + 1e-2 * rng.standard_normal(fpre.shape))
    tau_c = 0.8
    tf = train.fine_tau(tau_c, 3)
    post = lbm.bgk_collide(fpre, tf)
    a = train.restrict_forced(fpre, 3, tf, tau_c, 0.0)
    b = train.restrict(np.roll(post, (-1, -1), axis=(1, 2)), 3, tf, tau_c)
    assert a.shape == (9, 4, 3)
    assert np.allclose(a, b, rtol=0, atol=1e-15)


def test_restrict_forced_injects_forced_moments():
    """rho is injected and the coarse state's time-level velocity
    (sum f* e - F_c/2) / rho equals the fine node's forced velocity, with
    F_c = 3 F_f."""
    from oracle import channel
    rng = np.random.default_rng(32)
    f = lbm.equilibrium(np.ones((6, 9)), np.full((6, 9), 0.02), np.zeros((6, 9)))
    f = channel.channel_run(f * (1 + 1e-2 * rng.standard_normal(f.shape)), 0.9, 1e-4, 5)
    fpre = channel.stream_pull_walls(f)
    c = train.restrict_forced(fpre, 3, 0.9, 0.6333333333333333, 1e-4)
    rho_f, ux_f, uy_f = channel.moments_forced(fpre[:, 1::3, 1::3], 1e-4)
    rho_c, jx, jy = lbm.moments(c)
    assert np.allclose(rho_c, rho_f, rtol=1e-14, atol=0)
    assert np.allclose(jx - 1.5e-4 / rho_c, ux_f, rtol=0, atol=1e-15)
    assert np.allclose(jy, uy_f, rtol=0, atol=1e-15)


def test_restrict_forced_steady_channel_converges_at_second_order():
    """The steady channel on a 3x finer lattice, restricted, approaches the
    coarse lattice's steady channel as H grows: the gap in the
    non-equilibrium part shrinks at second order (the wall slip's order)."""
    from oracle import channel

    def steady(ny, nx, tau, g):
        f = lbm.equilibrium(np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))
        return channel.channel_run(f, tau, g, int(14 * ny * ny / (np.pi ** 2 * lbm.viscosity(tau))) + 300)

    def neq(f, g):
        rho, jx, jy = lbm.moments(f)
        return f - lbm.equilibrium(rho, jx - g / 2 / rho, jy)

    tau_c, umax = 0.6, 0.02
    gaps = []
    for h in (4, 8):
        gc = 8 * lbm.viscosity(tau_c) * umax / h ** 2
        tf = train.fine_tau(tau_c, 3)
        fc = steady(h, 1, tau_c, gc)
        ff = steady(3 * h, 3, tf, gc / 3)
        r = train.restrict_forced(channel.stream_pull_walls(ff), 3, tf, tau_c, gc / 3)
        a = neq(fc, gc)
        gaps.append(np.abs(neq(r, gc) - a).max() / np.abs(a).max())
    assert gaps[0] < 0.02 and 3.5 < gaps[0] / gaps[1] < 4.5, gaps


def test_channel_pair_is_close_to_one_coarse_channel_step():
    """A restricted channel pair (start-up from rest) is consistent with the
    coarse lattice away from the walls: one coarse BGK channel step from the
    input lands near the target in the interior rows, over 10x nearer than
    the input itself; in the rows next to the walls the coarse step misses
    by the difference between the two lattices' bounce-back slips (the
    error a trained collision can remove)."""
    from oracle import channel
    tau_c, ny, nx = 0.7, 8, 2
    gc = 8 * lbm.viscosity(tau_c) * 0.03 / ny ** 2
    f_in, f_tg = train.channel_pair(ny, nx, tau_c, gc, 30)
    assert f_in.shape == f_tg.shape == (9, ny, nx)
    step = channel.channel_step(f_in, tau_c, gc)
    inner = slice(1, ny - 1)
    err = np.abs(step - f_tg)[:, inner].max()
    assert err < 0.1 * np.abs(f_in - f_tg)[:, inner].max()
    assert np.abs(step - f_tg)[:, [0, ny - 1]].max() > 10 * err


# ---- the K-step rollout loss (reverse mode through the dynamics) --------------------
def test_stream_adjoint_is_the_transpose():
    """<stream(f), g> = <f, stream_adjoint(g)> for random f, g (periodic
    wrap included), and the adjoint undoes the pull."""
    rng = np.random.default_rng(41)
    f = rng.standard_normal((9, 5, 7))
    g = rng.standard_normal((9, 5, 7))
    a = float(np.sum(lbm.stream_pull(f) * g))
    b = float(np.sum(f * lbm.stream_pull_adjoint(g)))
    assert abs(a - b) <= 1e-12 * abs(a)
    assert np.allclose(lbm.stream_pull_adjoint(lbm.stream_pull(f)), f, rtol=0, atol=0)


@pytest.mark.parametrize("variant", [0, 2, 4])
def test_collide_adjoint_matches_central_differences(variant):
    """The explicit part of Eq. 3's reverse mode: with y held fixed,
    <g, d f*(f_pre + h d)/dh> equals <collide_adjoint df, d>, and dL/dy
    equals the directional derivative in y."""
    from oracle import gnn
    rng = np.random.default_rng(42 + variant)
    f = lbm.tgv_init(4, 3, 1.0, 0.06, 2 * np.pi / 4, 2 * np.pi / 3)
    f = f * (1 + 2e-2 * rng.standard_normal(f.shape))
    p = gnn.unpack(inputs.xavier_params(3, s_df=1e-2, variant=variant))
    y = rng.standard_normal((12, 10))
    g = rng.standard_normal((9, 12))
    dy, df = train.collide_adjoint(f, y, 0.7, p, g)
    J = lambda ff, yy: float(np.sum(g * gnn.gnn_collide(ff, yy, 0.7, p).reshape(9, -1)))
    d = rng.standard_normal(f.shape)
    h = 1e-6
    fd = (J(f + h * d, y) - J(f - h * d, y)) / (2 * h)
    assert abs(fd - float(np.sum(df * d.reshape(9, -1)))) <= 1e-7 * abs(fd)
    dd = rng.standard_normal(y.shape)
    fd = (J(f, y + h * dd) - J(f, y - h * dd)) / (2 * h)
    an = float(np.sum(dy * dd))
    assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-12)


def test_rollout_loss_one_step_is_eq4():
    """K = 1: the rollout loss and gradient are Eq. 4's (collide_loss with
    the network's backward)."""
    from oracle import gnn
    f0 = lbm.tgv_init(4, 4, 1.0, 0.05, 2 * np.pi / 4, 2 * np.pi / 4)
    f0 = f0 * inputs.perturbation(f0.shape, 5, 1e-2)
    tg = lbm.bgk_step(f0, 0.8) * inputs.perturbation(f0.shape, 6, 1e-3)
    theta = inputs.xavier_params(9, s_df=1e-2, bias_scale=0.1)
    loss, grads, _ = train.rollout_loss(f0, [tg], theta, 0.8)
    p = gnn.unpack(theta)
    fpre = lbm.stream_pull(f0)
    y, cache = gnn.forward(fpre, p)
    l1, dy, _ = gnn.collide_loss(fpre, y, 0.8, tg, p)
    g1 = gnn.pack_grads(gnn.backward(dy, cache, p)[0])
    assert abs(loss - l1) <= 1e-14 * l1
    assert np.allclose(grads, g1, rtol=1e-10, atol=1e-18)


@pytest.mark.parametrize("K", [2, 3])
def test_rollout_gradient_matches_central_differences(K):
    """K-step rollout: the reverse-mode gradient w.r.t. every parameter
    tensor (directional derivatives) and w.r.t. the initial state agrees
    with central differences of the loss in FP64."""
    from oracle import gnn
    rng = np.random.default_rng(50 + K)
    f0 = lbm.tgv_init(4, 4, 1.0, 0.06, 2 * np.pi / 4, 2 * np.pi / 4)
    f0 = f0 * (1 + 2e-2 * rng.standard_normal(f0.shape))
    tgs = [lbm.bgk_run(f0, 0.75, k + 1) * (1 + 1e-3 * rng.standard_normal(f0.shape))
           for k in range(K)]
    p = gnn.unpack(inputs.xavier_params(11, s_df=1e-2, bias_scale=0.1))
    loss, grads, df0 = train.rollout_loss(f0, tgs, p, 0.75)
    L = lambda pp, ff: train.rollout_loss(ff, tgs, pp, 0.75)[0]
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
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


def test_restrict_forced_factor_one_is_one_channel_collision():
    """m = 1 (tau_f = tau_c): restricting the pulled state is one collision
    with Guo's source, (1 - 1/tau)(N - P) + P = (1 - 1/tau) N + P / tau with
    P / tau = (1 - 1/(2 tau)) S, i.e. exactly one BGK channel step."""
    from oracle import channel
    rng = np.random.default_rng(61)
    f = lbm.equilibrium(np.ones((5, 4)), np.full((5, 4), 0.03), np.zeros((5, 4)))
    f = f * (1 + 1e-2 * rng.standard_normal(f.shape))
    for tau, g in ((0.6, 2e-4), (1.3, -5e-4)):
        a = train.restrict_forced(channel.stream_pull_walls(f), 1, tau, tau, g)
        assert np.allclose(a, channel.channel_step(f, tau, g), rtol=0, atol=1e-16)
