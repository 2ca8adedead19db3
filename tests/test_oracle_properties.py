"""Property-based pins of the FP64 oracle (no GPU): facts that hold for every
lattice size, state and relaxation time, checked on random draws.

  * Eq. 2: the moments of f^eq are exactly rho, rho u and the momentum flux
    rho (c_s^2 I + u u) (the D2Q9 weights' isotropy up to 4th order);
  * Fig. 1 streaming is a permutation of each population plane;
  * Eq. 1 with streaming conserves the domain's mass and momentum;
  * the network with every trainable value zero gives tau_adj = 1 and
    Delta f = 0, so Eq. 3 reduces to Eq. 1 exactly;
  * the GNN-LBM step commutes with periodic translations of the lattice (the
    message passing uses only relative neighbours, Sec. 2.2);
  * the conserving projection of Delta f (this library's option) leaves no
    component along 1, e_x, e_y and is idempotent;
  * the forced channel restriction (the library's reading of Sec. 2.4 for
    the flow of Sec. 3.1) injects rho and the time-level velocity
    (sum f* e - F_c/2)/rho with F_c = m F_f, for any state, odd m, tau and
    force, and without force equals the periodic restriction of the
    collided state;
  * the channel step (halfway bounce-back, Guo forcing) conserves the
    domain's mass and commutes with the mirror about the centre line and
    with shifts along the channel;
  * the K-step rollout loss's reverse-mode gradient is its derivative along
    any direction of the parameters and of the initial state.
"""
import numpy as np
import pytest

from oracle import gnn, lbm
from paper_2504_14494_gb300 import inputs

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
given, settings = hyp.given, hyp.settings

SETTINGS = settings(max_examples=25, deadline=None, derandomize=True)
sizes = st.integers(min_value=1, max_value=7)
seeds = st.integers(min_value=0, max_value=2 ** 31 - 1)


def _state(nx, ny, seed, amp=0.05, u0=0.06):
    rng = np.random.default_rng(seed)
    rho = 1.0 + amp * rng.uniform(-1, 1, (ny, nx))
    ux = u0 * rng.uniform(-1, 1, (ny, nx))
    uy = u0 * rng.uniform(-1, 1, (ny, nx))
    f = lbm.equilibrium(rho, ux, uy)
    return f * (1.0 + 0.1 * amp * rng.uniform(-1, 1, f.shape))


@SETTINGS
@given(seed=seeds)
def test_equilibrium_moments_for_random_states(seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0, 16)
    ux, uy = rng.uniform(-0.2, 0.2, 16), rng.uniform(-0.2, 0.2, 16)
    feq = lbm.equilibrium(rho, ux, uy)
    e = lbm.E.astype(np.float64)
    assert np.allclose(feq.sum(axis=0), rho, rtol=1e-13)
    assert np.allclose((e[:, 0, None] * feq).sum(axis=0), rho * ux, rtol=1e-12, atol=1e-15)
    assert np.allclose((e[:, 1, None] * feq).sum(axis=0), rho * uy, rtol=1e-12, atol=1e-15)
    u = (ux, uy)
    for a in range(2):
        for b in range(2):
            flux = (e[:, a, None] * e[:, b, None] * feq).sum(axis=0)
            want = rho * (lbm.CS2 * (a == b) + u[a] * u[b])
            assert np.allclose(flux, want, rtol=1e-12, atol=1e-15), (a, b)


@SETTINGS
@given(nx=sizes, ny=sizes, seed=seeds)
def test_streaming_permutes_each_plane(nx, ny, seed):
    f = _state(nx, ny, seed)
    g = lbm.stream_pull(f)
    for q in range(lbm.Q):
        assert np.array_equal(np.sort(g[q].ravel()), np.sort(f[q].ravel()))
    # shifting by e_q is undone by shifting back
    back = np.stack([np.roll(g[q], (-lbm.E[q, 1], -lbm.E[q, 0]), axis=(0, 1))
                     for q in range(lbm.Q)])
    assert np.array_equal(back, f)


@SETTINGS
@given(nx=sizes, ny=sizes, seed=seeds, tau=st.floats(min_value=0.505, max_value=2.0))
def test_bgk_step_conserves_mass_and_momentum(nx, ny, seed, tau):
    f = _state(nx, ny, seed)
    t0 = lbm.totals(f)
    t1 = lbm.totals(lbm.bgk_step(f, tau))
    assert abs(t1[0] - t0[0]) <= 1e-13 * t0[0]
    assert abs(t1[1] - t0[1]) <= 1e-13 * t0[0] and abs(t1[2] - t0[2]) <= 1e-13 * t0[0]


@SETTINGS
@given(nx=sizes, ny=sizes, seed=seeds, tau=st.floats(min_value=0.505, max_value=2.0))
def test_zero_network_step_is_the_bgk_step(nx, ny, seed, tau):
    f = _state(nx, ny, seed)
    theta = inputs.zero_params(s_df=1e-2)
    assert np.allclose(gnn.gnn_step(f, theta, tau), lbm.bgk_step(f, tau), rtol=1e-14,
                       atol=1e-16)


@SETTINGS
@given(nx=st.integers(2, 6), ny=st.integers(2, 6), seed=seeds, dx=st.integers(0, 5),
       dy=st.integers(0, 5))
def test_gnn_step_commutes_with_translations(nx, ny, seed, dx, dy):
    f = _state(nx, ny, seed)
    theta = inputs.xavier_params(seed % 1000, s_df=1e-2, bias_scale=0.1)
    shift = (dy % ny, dx % nx)
    a = gnn.gnn_step(np.roll(f, shift, axis=(1, 2)), theta, 0.7)
    b = np.roll(gnn.gnn_step(f, theta, 0.7), shift, axis=(1, 2))
    assert np.allclose(a, b, rtol=1e-12, atol=1e-15)


@SETTINGS
@given(seed=seeds)
def test_conserving_projection(seed):
    rng = np.random.default_rng(seed)
    df = rng.standard_normal((9, 11))
    p = gnn.conserve(df)
    e = lbm.E.astype(np.float64)
    assert np.allclose(p.sum(axis=0), 0.0, atol=1e-13)
    assert np.allclose((e[:, 0, None] * p).sum(axis=0), 0.0, atol=1e-13)
    assert np.allclose((e[:, 1, None] * p).sum(axis=0), 0.0, atol=1e-13)
    assert np.allclose(gnn.conserve(p), p, atol=1e-13)
    # the removed part lies in span{1, e_x, e_y}
    basis = np.stack([np.ones(9), e[:, 0], e[:, 1]], axis=1)
    coef, *_ = np.linalg.lstsq(basis, df - p, rcond=None)
    assert np.allclose(basis @ coef, df - p, atol=1e-12)


@SETTINGS
@given(nyc=sizes, nxc=sizes, m=st.sampled_from([1, 3, 5]), seed=seeds,
       tau_c=st.floats(min_value=0.52, max_value=1.8),
       gf=st.floats(min_value=-1e-3, max_value=1e-3))
def test_forced_restriction_injects_moments(nyc, nxc, m, seed, tau_c, gf):
    from oracle import channel, train
    f = _state(m * nxc, m * nyc, seed)
    tf = train.fine_tau(tau_c, m)
    c = train.restrict_forced(f, m, tf, tau_c, gf)
    o = (m - 1) // 2
    rho_f, ux_f, uy_f = channel.moments_forced(f[:, o::m, o::m], gf)
    rho_c, jx, jy = lbm.moments(c)
    assert np.allclose(rho_c, rho_f, rtol=1e-13, atol=0)
    assert np.allclose(jx - 0.5 * m * gf / rho_c, ux_f, rtol=0, atol=1e-14)
    assert np.allclose(jy, uy_f, rtol=0, atol=1e-14)
    if m > 1:
        post = lbm.bgk_collide(f, tf)
        a = train.restrict_forced(f, m, tf, tau_c, 0.0)
        b = train.restrict(np.roll(post, (-o, -o), axis=(1, 2)), m, tf, tau_c)
        assert np.allclose(a, b, rtol=0, atol=1e-14)


MIRROR_Y = [0, 1, 4, 3, 2, 8, 7, 6, 5]   # e_i -> e_i with e_y negated


@SETTINGS
@given(ny=sizes, nx=sizes, seed=seeds, tau=st.floats(min_value=0.51, max_value=2.0),
       gx=st.floats(min_value=-1e-3, max_value=1e-3), shift=st.integers(0, 6))
def test_channel_step_conserves_mass_and_keeps_the_channel_symmetries(ny, nx, seed, tau, gx,
                                                                      shift):
    from oracle import channel
    f = _state(nx, ny, seed)
    g = channel.channel_step(f, tau, gx)
    assert abs(g.sum() - f.sum()) <= 1e-12 * f.sum()
    # mirror about the channel's centre line (walls swap places)
    mirror = lambda a: a[MIRROR_Y, ::-1, :]
    assert np.allclose(channel.channel_step(mirror(f), tau, gx), mirror(g), rtol=0, atol=1e-15)
    # periodic in x
    assert np.allclose(channel.channel_step(np.roll(f, shift, axis=2), tau, gx),
                       np.roll(g, shift, axis=2), rtol=0, atol=1e-15)


@settings(max_examples=10, deadline=None, derandomize=True)
@given(nx=st.integers(2, 4), ny=st.integers(2, 4), K=st.integers(1, 2), seed=seeds,
       tau=st.floats(min_value=0.55, max_value=1.2))
def test_rollout_gradient_is_the_derivative_of_the_rollout_loss(nx, ny, K, seed, tau):
    """The K-step rollout loss's reverse-mode gradient (through Eq. 3, the
    network and streaming) gives its directional derivative along a random
    direction of all parameters and of the initial state, for any small
    lattice, K and tau (central differences in FP64)."""
    from oracle import train
    rng = np.random.default_rng(seed)
    f0 = _state(nx, ny, seed)
    tgs = [_state(nx, ny, seed + 1 + k) for k in range(K)]
    p = gnn.unpack(inputs.xavier_params(seed % 1000, s_df=1e-2, bias_scale=0.1))
    loss, grads, df0 = train.rollout_loss(f0, tgs, p, tau)
    d = {name: rng.standard_normal(shape) for name, shape in gnn.SHAPES}
    an = float(np.dot(grads, np.concatenate([d[name].ravel() for name, _ in gnn.SHAPES])))
    h = 1e-6
    q1 = {k: (v + h * d[k] if k in d else v) for k, v in p.items()}
    q2 = {k: (v - h * d[k] if k in d else v) for k, v in p.items()}
    fd = (train.rollout_loss(f0, tgs, q1, tau)[0] - train.rollout_loss(f0, tgs, q2, tau)[0]) / (2 * h)
    assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-9), (fd, an)
    e = rng.standard_normal(f0.shape) * 1e-2
    fd = (train.rollout_loss(f0 + 1e-4 * e, tgs, p, tau)[0]
          - train.rollout_loss(f0 - 1e-4 * e, tgs, p, tau)[0]) / 2e-4
    an = float(np.sum(df0 * e))
    # the state step moves the loss by ~1e-9 of itself: round-off ~1e-6 of fd
    assert abs(fd - an) <= 2e-5 * max(abs(an), 1e-12), (fd, an)
