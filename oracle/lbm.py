"""FP64 oracle for the plain D2Q9 BGK lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
  * Sec. 2.1, Eq. 1  -- BGK update  f_i(x+e_i, t+1) = f_i - (f_i - f_i^eq)/tau.
  * Sec. 2.1, Eq. 2  -- second-order equilibrium
        f_i^eq = rho w_i [1 + e_i.u/c_s^2 + (e_i.u)^2/(2 c_s^4) - u.u/(2 c_s^2)].
  * Fig. 1           -- loop order: macroscopic variables, collision, streaming,
                        boundary conditions (periodic wrap here).
  * Sec. 3.2         -- Taylor-Green vortex benchmark and its analytic decay.
  * Sec. 3.3, Eq. 6  -- convergence rate alpha = log(E1/E2)/log(h1/h2).

Readings of passages the paper leaves open:
  * D2Q9 velocity order and weights (Sec. 2.1 names w_i and c_s but lists no
    values): e_0=(0,0); e_1..4=(1,0),(0,1),(-1,0),(0,-1);
    e_5..8=(1,1),(-1,1),(-1,-1),(1,-1); w = 4/9, 1/9 (x4), 1/36 (x4); c_s^2=1/3.
  * Array layout: f[q, y, x] (x fastest), q-major, node coordinates integer.
  * Stored state: the POST-collision populations f*(., n).  One step pulls
    f_i(x) = f*_i(x - e_i) (streaming), takes moments, collides, and stores
    f*(., n+1).  Initialising with f^eq is consistent, since f^eq is a fixed
    point of the collision.
  * Periodic wrap in x and y (the TGV benchmark is periodic).
  * TGV initial field (Sec. 3.2 gives no formula):
        u_x =  u0 cos(k x) sin(k y),  u_y = -u0 sin(k x) cos(k y),
    rho = rho0 (uniform) or, optionally, the pressure-consistent
    rho = rho0 (1 - 3/4 u0^2 (cos 2kx + cos 2ky)).
  * Analytic decay: u(t) = u(0) exp(-2 nu k^2 t), nu = c_s^2 (tau - 1/2);
    kinetic energy E(t) = E(0) exp(-4 nu k^2 t).
  * "L2 velocity error" (Sec. 3.2, Table 2, undefined in the paper): the
    relative error sqrt(sum |u - u_a|^2 / sum |u_a|^2).
"""
import numpy as np

# --- D2Q9 lattice (Sec. 2.1) --------------------------------------------------
E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1],
              [1, 1], [-1, 1], [-1, -1], [1, -1]], dtype=np.int64)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=np.float64)
CS2 = 1.0 / 3.0
Q = 9


def equilibrium(rho, ux, uy):
    """Eq. 2: f_i^eq for every direction.  rho, ux, uy: arrays of one shape S.

    Returns an array of shape (9,) + S in float64.
    """
    rho = np.asarray(rho, dtype=np.float64)
    ux = np.asarray(ux, dtype=np.float64)
    uy = np.asarray(uy, dtype=np.float64)
    uu = ux * ux + uy * uy
    feq = np.empty((Q,) + rho.shape, dtype=np.float64)
    for i in range(Q):
        eu = E[i, 0] * ux + E[i, 1] * uy
        feq[i] = rho * W[i] * (1.0 + eu / CS2 + eu * eu / (2.0 * CS2 * CS2)
                               - uu / (2.0 * CS2))
    return feq


def moments(f):
    """Macroscopic variables (Fig. 1, 'Compute macroscopic variables').

    rho = sum_i f_i,  rho u = sum_i f_i e_i.  f: (9, ...) -> (rho, ux, uy).
    """
    f = np.asarray(f, dtype=np.float64)
    rho = f.sum(axis=0)
    jx = np.zeros_like(rho)
    jy = np.zeros_like(rho)
    for i in range(Q):
        jx = jx + E[i, 0] * f[i]
        jy = jy + E[i, 1] * f[i]
    return rho, jx / rho, jy / rho


def stream_pull(fpost):
    """Streaming with periodic wrap, written as a pull by explicit indexing.

    f_i(x, y) <- f*_i((x - e_ix) mod nx, (y - e_iy) mod ny) for f[q, y, x].
    This is Fig. 1's streaming step f_i(x + e_i, t+1) = f_i^*(x, t).
    """
    fpost = np.asarray(fpost, dtype=np.float64)
    _, ny, nx = fpost.shape
    out = np.empty_like(fpost)
    xs = np.arange(nx)
    ys = np.arange(ny)
    for i in range(Q):
        src_x = (xs - E[i, 0]) % nx
        src_y = (ys - E[i, 1]) % ny
        out[i] = fpost[i][src_y[:, None], src_x[None, :]]
    return out


def stream_pull_adjoint(g):
    """Adjoint of ``stream_pull`` (a linear map): with out_i(x) = f_i(x - e_i)
    periodic, <stream_pull(f), g> = <f, stream_pull_adjoint(g)> for all f, g,
    so the adjoint pushes back: result_i(x) = g_i(x + e_i)."""
    g = np.asarray(g, np.float64)
    out = np.empty_like(g)
    for i in range(Q):
        out[i] = np.roll(g[i], shift=(-int(E[i, 1]), -int(E[i, 0])), axis=(0, 1))
    return out


def bgk_collide(f, tau):
    """Eq. 1 (Fig. 1 'Standard BGK Collision'): f* = f - (f - f^eq)/tau."""
    rho, ux, uy = moments(f)
    feq = equilibrium(rho, ux, uy)
    return f - (f - feq) / tau


def bgk_step(fpost, tau):
    """One full BGK step on the stored post-collision state.

    Pull-stream (periodic), then moments, equilibrium and the BGK relaxation;
    returns the new post-collision state f*(., n+1).
    """
    return bgk_collide(stream_pull(fpost), tau)


def bgk_run(fpost, tau, nsteps):
    f = np.asarray(fpost, dtype=np.float64)
    for _ in range(nsteps):
        f = bgk_step(f, tau)
    return f


# --- Taylor-Green vortex (Sec. 3.2) --------------------------------------------
def tgv_velocity(nx, ny, u0, kx, ky):
    """Initial TGV velocity at integer node coordinates (reading in header)."""
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    ux = u0 * np.cos(kx * x) * np.sin(ky * y)
    uy = -u0 * np.sin(kx * x) * np.cos(ky * y)
    return ux, uy


def tgv_density(nx, ny, rho0, u0, kx, ky, pressure_consistent=False):
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    if pressure_consistent:
        return rho0 * (1.0 - 0.75 * u0 * u0 * (np.cos(2 * kx * x) + np.cos(2 * ky * y)))
    return np.full((ny, nx), float(rho0))


def tgv_init(nx, ny, rho0, u0, kx, ky, pressure_consistent=False):
    """f = f^eq(rho(x), u_TGV(x, 0)) on an ny x nx lattice: shape (9, ny, nx)."""
    ux, uy = tgv_velocity(nx, ny, u0, kx, ky)
    rho = tgv_density(nx, ny, rho0, u0, kx, ky, pressure_consistent)
    return equilibrium(rho, ux, uy)


def viscosity(tau):
    """Lattice kinematic viscosity of BGK: nu = c_s^2 (tau - 1/2)."""
    return CS2 * (tau - 0.5)


def tgv_analytic_velocity(nx, ny, u0, kx, ky, tau, t):
    """Closed-form TGV decay u(t) = u(0) exp(-nu (kx^2 + ky^2) t)."""
    ux, uy = tgv_velocity(nx, ny, u0, kx, ky)
    decay = np.exp(-viscosity(tau) * (kx * kx + ky * ky) * t)
    return ux * decay, uy * decay


def velocity_l2_error(ux, uy, ux_a, uy_a):
    """Relative L2 velocity error sqrt(sum|u-u_a|^2 / sum|u_a|^2)."""
    num = np.sum((ux - ux_a) ** 2 + (uy - uy_a) ** 2)
    den = np.sum(ux_a ** 2 + uy_a ** 2)
    return float(np.sqrt(num / den))


def totals(f):
    """Domain totals in FP64: mass, momentum x, momentum y, kinetic energy
    E = 1/2 sum rho |u|^2 = 1/2 sum |rho u|^2 / rho, and the number of nodes
    holding a non-finite population (those nodes are left out of the sums)."""
    f = np.asarray(f, dtype=np.float64)
    bad = ~np.all(np.isfinite(f), axis=0)
    f = np.where(bad[None], 0.0, f)
    rho = f.sum(axis=0)
    jx = sum(E[i, 0] * f[i] for i in range(Q))
    jy = sum(E[i, 1] * f[i] for i in range(Q))
    energy = 0.5 * np.sum(np.where(bad, 0.0, (jx * jx + jy * jy) / np.where(bad, 1.0, rho)))
    nonfinite = int(np.count_nonzero(bad))
    return np.array([rho.sum(), jx.sum(), jy.sum(), energy, float(nonfinite)])


def convergence_rate(e1, e2, h1, h2):
    """Eq. 6: alpha = log(E1/E2) / log(h1/h2)."""
    return float(np.log(e1 / e2) / np.log(h1 / h2))
