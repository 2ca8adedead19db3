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
