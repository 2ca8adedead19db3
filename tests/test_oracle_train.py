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
