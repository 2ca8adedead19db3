"""Pins of the FP64 LBM oracle against facts the paper and the mathematics fix
(no GPU).  Each test names the passage it pins."""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import lbm
from paper_2504_14494_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_d2q9_lattice_identities():
    """Sec. 2.1: the weights w_i and sound speed c_s of D2Q9 satisfy the
    isotropy conditions up to 4th order (textbook D2Q9)."""
    e = lbm.E.astype(np.float64)
    w = lbm.W
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(w @ e, 0.0, atol=1e-15)
    m2 = np.einsum("i,ia,ib->ab", w, e, e)
    assert np.allclose(m2, lbm.CS2 * np.eye(2), atol=1e-15)
    m3 = np.einsum("i,ia,ib,ic->abc", w, e, e, e)
    assert np.allclose(m3, 0.0, atol=1e-15)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    d = np.eye(2)
    iso = lbm.CS2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                          + np.einsum("ad,bc->abcd", d, d))
    assert np.allclose(m4, iso, atol=1e-15)
    # opposite directions come in pairs with equal weight
    for i in range(9):
        j = [k for k in range(9) if (lbm.E[k] == -lbm.E[i]).all()]
        assert len(j) == 1 and lbm.W[j[0]] == lbm.W[i]


def test_equilibrium_moments():
    """Eq. 2: f^eq reproduces rho, rho u and the momentum flux
    rho (c_s^2 I + u u) exactly (closed form of the 2nd-order Maxwellian)."""
    rng = np.random.default_rng(1)
    rho = 1.0 + 0.1 * rng.standard_normal(50)
    ux = 0.1 * rng.standard_normal(50)
    uy = 0.1 * rng.standard_normal(50)
    feq = lbm.equilibrium(rho, ux, uy)
    e = lbm.E.astype(np.float64)
    assert np.allclose(feq.sum(0), rho, rtol=1e-14, atol=0)
    assert np.allclose(np.einsum("in,i->n", feq, e[:, 0]), rho * ux, rtol=0, atol=1e-15)
    assert np.allclose(np.einsum("in,i->n", feq, e[:, 1]), rho * uy, rtol=0, atol=1e-15)
    pxx = np.einsum("in,i->n", feq, e[:, 0] * e[:, 0])
    pxy = np.einsum("in,i->n", feq, e[:, 0] * e[:, 1])
    pyy = np.einsum("in,i->n", feq, e[:, 1] * e[:, 1])
    assert np.allclose(pxx, rho * (lbm.CS2 + ux * ux), rtol=1e-14)
    assert np.allclose(pxy, rho * ux * uy, rtol=0, atol=1e-15)
    assert np.allclose(pyy, rho * (lbm.CS2 + uy * uy), rtol=1e-14)
    # at rest f^eq = rho w_i
    assert np.allclose(lbm.equilibrium(np.array([2.0]), np.array([0.0]), np.array([0.0]))[:, 0],
                       2.0 * lbm.W, rtol=1e-15)


def test_equilibrium_is_fixed_point_of_bgk():
    """Eq. 1: the BGK relaxation leaves f^eq unchanged."""
    f = lbm.tgv_init(8, 6, 1.0, 0.05, 2 * np.pi / 8, 2 * np.pi / 6)
    assert np.allclose(lbm.bgk_collide(f, 0.7), f, rtol=0, atol=1e-15)


def test_streaming_moves_a_delta_along_e_i():
    """Fig. 1 streaming f_i(x + e_i, t+1) = f*_i(x, t): a unit population at
    (x0, y0) in direction i arrives at (x0 + e_ix, y0 + e_iy) mod (nx, ny),
    including across the periodic edges."""
    nx, ny = 5, 4
    for i, (x0, y0) in itertools.product(range(9), [(0, 0), (4, 3), (2, 1)]):
        f = np.zeros((9, ny, nx))
        f[i, y0, x0] = 1.0
        g = lbm.stream_pull(f)
        ys, xs = np.nonzero(g[i])
        assert (xs[0], ys[0]) == ((x0 + lbm.E[i, 0]) % nx, (y0 + lbm.E[i, 1]) % ny)
        assert g.sum() == 1.0


def test_bgk_conserves_mass_and_momentum_1000_steps():
    """Eq. 1 with Eq. 2 conserves mass and momentum exactly; over 1000 FP64
    steps of the 64^2 TGV (tau=0.8, u0=0.01) the drift stays below 1e-12
    relative (momentum normalised by M u0, since the TGV total is 0)."""
    n, u0 = 64, 0.01
    k = 2 * np.pi / n
    f = lbm.tgv_init(n, n, 1.0, u0, k, k)
    # break the symmetry so that momentum conservation is not trivial
    f = f * inputs.perturbation(f.shape, 7, 1e-3)
    t0 = lbm.totals(f)
    g = lbm.bgk_run(f, 0.8, 1000)
    t1 = lbm.totals(g)
    mass = t0[0]
    assert abs(t1[0] - mass) / mass < 1e-12
    assert abs(t1[1] - t0[1]) / (mass * u0) < 1e-12
    assert abs(t1[2] - t0[2]) / (mass * u0) < 1e-12
    assert t1[4] == 0


def test_tgv_decay_closed_form():
    """Sec. 3.2 TGV: the velocity decays as u0 exp(-2 nu k^2 t) with
    nu = (tau - 1/2)/3.  At the 64^2, tau=0.8, u0=0.01 workload the oracle
    stays within 2e-3 relative L2 of the closed form after 1000 steps, and the
    kinetic-energy decay rate matches 4 nu k^2 to 0.5%."""
    n, u0, tau = 64, 0.01, 0.8
    k = 2 * np.pi / n
    f = lbm.tgv_init(n, n, 1.0, u0, k, k)
    e_prev = lbm.totals(f)[3]
    f = lbm.bgk_run(f, tau, 500)
    e500 = lbm.totals(f)[3]
    f = lbm.bgk_run(f, tau, 500)
    e1000 = lbm.totals(f)[3]
    rho, ux, uy = lbm.moments(f)
    ua = lbm.tgv_analytic_velocity(n, n, u0, k, k, tau, 1000)
    err = lbm.velocity_l2_error(ux, uy, *ua)
    assert err < 2e-3
    rate = np.log(e500 / e1000) / 500.0
    assert abs(rate / (4 * lbm.viscosity(tau) * k * k) - 1.0) < 5e-3
    assert e_prev > e500 > e1000


def test_convergence_rate_second_order():
    """Sec. 3.3 / Eq. 6: under diffusive scaling (tau fixed, u0 ~ 1/N,
    steps ~ N^2) the TGV velocity error of LBM converges at alpha ~ 2.
    Uses the pressure-consistent initial density (the uniform-density start
    adds an O(Ma) acoustic transient that masks the rate)."""
    tau = 0.8
    errs = []
    ns = [32, 64, 128]
    for n in ns:
        k = 2 * np.pi / n
        u0 = 0.64 / n
        steps = n * n // 16
        f = lbm.tgv_init(n, n, 1.0, u0, k, k, pressure_consistent=True)
        f = lbm.bgk_run(f, tau, steps)
        rho, ux, uy = lbm.moments(f)
        errs.append(lbm.velocity_l2_error(ux, uy, *lbm.tgv_analytic_velocity(n, n, u0, k, k, tau, steps)))
    for i in range(2):
        alpha = lbm.convergence_rate(errs[i], errs[i + 1], 1.0 / ns[i], 1.0 / ns[i + 1])
        assert 1.9 < alpha < 2.1, (alpha, errs)


def test_pressure_consistent_density():
    """TGV pressure p = p0 - rho0 u0^2/4 (cos 2kx + cos 2ky), rho = p/c_s^2:
    its mean is rho0 and its extremes rho0 (1 -+ 3/2 u0^2)."""
    n, u0 = 16, 0.1
    k = 2 * np.pi / n
    rho = lbm.tgv_density(n, n, 1.0, u0, k, k, True)
    assert abs(rho.mean() - 1.0) < 1e-15
    assert abs(rho.max() - (1 + 1.5 * u0 * u0)) < 1e-15
    assert abs(rho.min() - (1 - 1.5 * u0 * u0)) < 1e-15


def test_golden_tgv64_matches_stored():
    """Regression pin: the 64^2 TGV after 1000 steps reproduces the values
    written by tests/golden/make_golden.py (which calls only the oracle)."""
    with open(os.path.join(GOLDEN, "tgv64_bgk.json")) as fh:
        gold = json.load(fh)
    n = gold["n"]
    k = 2 * np.pi / n
    f = lbm.tgv_init(n, n, gold["rho0"], gold["u0"], k, k)
    f = lbm.bgk_run(f, gold["tau"], gold["steps"])
    rho, ux, uy = lbm.moments(f)
    err = lbm.velocity_l2_error(ux, uy, *lbm.tgv_analytic_velocity(n, n, gold["u0"], k, k,
                                                                   gold["tau"], gold["steps"]))
    assert abs(err - gold["l2_error"]) < 1e-12
    assert np.allclose(lbm.totals(f)[:4], gold["totals"][:4], rtol=1e-12, atol=1e-14)
