"""FP64 oracle for the plain BGK channel (Poiseuille) flow.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
  * Sec. 3.1, Eq. 5 -- Poiseuille flow between two walls driven by a constant
    force (pressure gradient) G: u(y) = G/(2 mu) y (H - y).
  * Fig. 1 "Apply Boundary Conditions" (no scheme is given).

Readings where the paper gives no scheme:
  * Channel along x, periodic in x; walls halfway between node rows, at
    y = -1/2 and y = ny - 1/2, so H = ny and the wall-distance of row y is
    y + 1/2.  Halfway bounce-back: a population that would be pulled from
    outside the channel is the opposite population of the same node after
    collision, f_i(x, y) = f*_opp(i)(x, y).
  * Body force F = (G, 0) per unit volume by Guo's scheme: the velocity is
    u = (sum f_i e_i + F/2) / rho, and the collision adds
    S_i = (1 - 1/(2 tau)) w_i [3 (e_i - u) + 9 (e_i . u) e_i] . F.
  * With rho = 1, mu = nu = (tau - 1/2)/3, the steady profile is
    u(y) = G/(2 nu) (y + 1/2) (ny - 1/2 - y).
  * Re = u_max H / nu with u_max = G H^2 / (8 nu).
  * Training loss of the channel network: Eq. 3 with Guo's source at the
    network's relaxation time, then Eq. 4 (``collide_loss_channel``); its
    K-step rollout form (``rollout_loss_channel``, the library's option
    beyond Eq. 4) differentiated through the walled pull, the forced
    collision and the walled network.
"""
import numpy as np

from . import lbm

OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])


def guo_term(ux, uy, gx, gy=0.0):
    """w_i [3 (e_i - u) + 9 (e_i . u) e_i] . F, Guo's source without its
    relaxation factor (1 - 1/(2 tau))."""
    s = np.empty((lbm.Q,) + np.broadcast(ux, uy, gx, gy).shape)
    for i in range(lbm.Q):
        ex, ey = lbm.E[i]
        eu = ex * ux + ey * uy
        tx = 3.0 * (ex - ux) + 9.0 * eu * ex
        ty = 3.0 * (ey - uy) + 9.0 * eu * ey
        s[i] = lbm.W[i] * (tx * gx + ty * gy)
    return s


def guo_source(ux, uy, tau, gx, gy=0.0):
    """Guo forcing term S_i for force (gx, gy) (per unit volume)."""
    return (1.0 - 0.5 / tau) * guo_term(ux, uy, gx, gy)


def moments_forced(f, gx, gy=0.0):
    """rho and the force-corrected velocity u = (sum f e + F/2)/rho."""
    rho = f.sum(axis=0)
    jx = sum(lbm.E[i, 0] * f[i] for i in range(lbm.Q))
    jy = sum(lbm.E[i, 1] * f[i] for i in range(lbm.Q))
    return rho, (jx + 0.5 * gx) / rho, (jy + 0.5 * gy) / rho


def stream_pull_walls(fpost):
    """Pull streaming, periodic in x, halfway bounce-back at y = -1/2 and
    y = ny - 1/2 (explicit indexing)."""
    _, ny, nx = fpost.shape
    out = np.empty_like(fpost)
    xs = np.arange(nx)
    ys = np.arange(ny)
    for i in range(lbm.Q):
        ex, ey = lbm.E[i]
        src_y = ys - ey
        inside = (src_y >= 0) & (src_y < ny)
        out[i][inside] = fpost[i][src_y[inside][:, None], ((xs - ex) % nx)[None, :]]
        out[i][~inside] = fpost[OPP[i]][~inside]
    return out


def stream_pull_walls_adjoint(g):
    """Adjoint of ``stream_pull_walls`` (a linear map, periodic in x with
    halfway bounce-back): <stream_pull_walls(f), g> = <f, result> for all f.
    A pulled value from inside sends g back to its source node; a bounced
    value f_opp(i)(x) sends g_i(x) to population opp(i) of the same node."""
    g = np.asarray(g, np.float64)
    _, ny, nx = g.shape
    out = np.zeros_like(g)
    xs = np.arange(nx)
    ys = np.arange(ny)
    for i in range(lbm.Q):
        ex, ey = lbm.E[i]
        src_y = ys - ey
        inside = (src_y >= 0) & (src_y < ny)
        for y in ys[inside]:
            np.add.at(out[i], (y - ey, (xs - ex) % nx), g[i, y])
        for y in ys[~inside]:
            out[OPP[i], y] += g[i, y]
    return out


def channel_step(fpost, tau, gx):
    """One step: stream (walls), forced moments, BGK relaxation + Guo source."""
    f = stream_pull_walls(fpost)
    rho, ux, uy = moments_forced(f, gx)
    feq = lbm.equilibrium(rho, ux, uy)
    return f - (f - feq) / tau + guo_source(ux, uy, tau, gx)


def gnn_channel_step(fpost, theta, tau, gx):
    """One GNN-LBM step of the channel (Sec. 3.1 with the collision of Eq. 3;
    readings: the network runs on the channel's graph - periodic in x, no
    neighbour across a wall, whose messages are left out of the sum - with
    the force-corrected velocity among its features, and Guo's source uses
    the network's relaxation time tau tau_adj):
      f* = f - (f - f^eq)/(tau tau_adj) + S(tau tau_adj) + Delta f."""
    from . import gnn
    p = gnn.unpack(theta)
    f = stream_pull_walls(np.asarray(fpost, np.float64))
    q, ny, nx = f.shape
    y, _ = gnn.forward(f, p, walls=True, force_x=gx)
    tau_adj, df = gnn.heads(y, p)
    teff = (tau * tau_adj).reshape(ny, nx)
    rho, ux, uy = moments_forced(f, gx)
    feq = lbm.equilibrium(rho, ux, uy)
    return f - (f - feq) / teff + guo_source(ux, uy, teff, gx) + df.reshape(q, ny, nx)


def channel_run(fpost, tau, gx, nsteps):
    f = np.asarray(fpost, np.float64)
    for _ in range(nsteps):
        f = channel_step(f, tau, gx)
    return f


def poiseuille_profile(ny, tau, gx):
    """Eq. 5 in lattice units (rho = 1): u(y) = G/(2 nu) (y+1/2)(ny-1/2-y)."""
    y = np.arange(ny, dtype=np.float64)
    return gx / (2.0 * lbm.viscosity(tau)) * (y + 0.5) * (ny - 0.5 - y)


def collide_loss_channel(f_pre, y, tau, target, p, gx, node_weight=None):
    """The channel's form of Eq. 3 followed by Eq. 4 (the training loss of
    the channel network): with t = tau tau_adj,
        f_pred = f - (f - f^eq(rho, u))/t + (1 - 1/(2 t)) S(u) + Delta f,
    u the force-corrected velocity, S = guo_term(u, F); loss = mean over
    nodes x 9 of (f_pred - target)^2 (times node_weight, if given).
    tau, gx: scalars or per-node arrays (N,).  d f_pred / d t is
    ((f - f^eq) + S/2) / t^2.  Returns (loss, dL/dy (N, 10), f_pred (9, N))."""
    from . import gnn
    q = f_pre.shape[0]
    f = np.asarray(f_pre, np.float64).reshape(q, -1)
    gx = np.broadcast_to(np.asarray(gx, np.float64), f.shape[1:])
    rho, ux, uy = moments_forced(f, gx)
    feq = lbm.equilibrium(rho, ux, uy)
    src = guo_term(ux, uy, gx)
    t = np.asarray(target, np.float64).reshape(q, -1)
    tau_adj, df = gnn.heads(y, p)
    teff = tau * tau_adj
    f_pred = f - (f - feq) / teff + (1.0 - 0.5 / teff) * src + df
    n = f.size
    r = f_pred - t
    wn = 1.0 if node_weight is None else np.asarray(node_weight, np.float64)[None, :]
    loss = float(np.sum(wn * r * r) / n)
    dfs = 2.0 * wn * r / n
    dy = np.zeros_like(y)
    dy[:, 1:] = (p["s_df"] * (gnn.conserve(dfs) if p["variant"] & gnn.CONSERVATIVE
                              else dfs)).T
    dteff = np.sum(dfs * ((f - feq) + 0.5 * src), axis=0) / (teff * teff)
    s = gnn.sigmoid(y[:, 0])
    dy[:, 0] = 0.0 if p["variant"] & gnn.FIXED_TAU else dteff * tau * s * (1.0 - s)
    return loss, dy, f_pred


def collide_adjoint_channel(f_pre, y, tau, p, gx, g):
    """Reverse mode of the channel's Eq. 3 (Guo's source at t = tau tau_adj)
    given g = dL/df* (9, N): returns dL/dy (N, 10) and the part of
    dL/df_pre through the explicit f, f^eq(rho, u) and S(u), with the forced
    u = (j + F/2)/rho (so du/df_j = (e_j - u)/rho, as without force):
      d f*_i/d f_j = delta_ij (1 - 1/t) + (1/t) d f^eq_i/d f_j
                     + (1 - 1/(2t)) d S_i/d f_j,
      d S_i/d u = w_i [-3 F + 9 (e_i . F) e_i]."""
    from . import gnn
    q = lbm.Q
    f = np.asarray(f_pre, np.float64).reshape(q, -1)
    gxn = np.broadcast_to(np.asarray(gx, np.float64), f.shape[1:])
    rho, ux, uy = moments_forced(f, gxn)
    feq = lbm.equilibrium(rho, ux, uy)
    src = guo_term(ux, uy, gxn)
    g = np.asarray(g, np.float64).reshape(q, -1)
    tau_adj, _ = gnn.heads(y, p)
    t = tau * tau_adj
    dy = np.zeros_like(y)
    dy[:, 1:] = (p["s_df"] * (gnn.conserve(g) if p["variant"] & gnn.CONSERVATIVE else g)).T
    s = gnn.sigmoid(y[:, 0])
    dy[:, 0] = (0.0 if p["variant"] & gnn.FIXED_TAU
                else np.sum(g * ((f - feq) + 0.5 * src), axis=0) / (t * t) * tau * s * (1.0 - s))
    a = np.sum(g * feq, axis=0) / rho
    vx = np.zeros_like(rho)
    vy = np.zeros_like(rho)
    c = 1.0 - 0.5 / t
    for i in range(q):
        ex, ey = lbm.E[i]
        eu = ex * ux + ey * uy
        ef = ex * gxn
        vx += g[i] * lbm.W[i] * ((3.0 * ex + 9.0 * eu * ex - 3.0 * ux) / t
                                 + c * (-3.0 * gxn + 9.0 * ef * ex) / rho)
        vy += g[i] * lbm.W[i] * ((3.0 * ey + 9.0 * eu * ey - 3.0 * uy) / t
                                 + c * (9.0 * ef * ey) / rho)
    df = np.empty_like(f)
    for j in range(q):
        ex, ey = lbm.E[j]
        df[j] = g[j] * (1.0 - 1.0 / t) + a / t + vx * (ex - ux) + vy * (ey - uy)
    return dy, df


def rollout_loss_channel(f0, targets, theta, tau, gx):
    """The K-step rollout loss on the channel (walls, force gx): K GNN-LBM
    channel steps from f0, the mean over the steps of Eq. 4 against
    targets[k], and its gradient by reverse mode through the walled pull,
    the channel collision with Guo's source and the walled network.
    theta: a parameter vector or ``gnn.unpack``'s dict.  Returns (loss,
    packed dL/dtheta, dL/df0)."""
    from . import gnn
    p = theta if isinstance(theta, dict) else gnn.unpack(theta)
    K = len(targets)
    f = np.asarray(f0, np.float64)
    q, ny, nx = f.shape
    n = f.size
    tape = []
    loss = 0.0
    for k in range(K):
        fpre = stream_pull_walls(f)
        y, cache = gnn.forward(fpre, p, walls=True, force_x=gx)
        tau_adj, dfc = gnn.heads(y, p)
        teff = (tau * tau_adj).reshape(ny, nx)
        rho, ux, uy = moments_forced(fpre, gx)
        feq = lbm.equilibrium(rho, ux, uy)
        f = (fpre - (fpre - feq) / teff + guo_source(ux, uy, teff, gx)
             + dfc.reshape(q, ny, nx))
        r = f - np.asarray(targets[k], np.float64)
        loss += float(np.sum(r * r)) / (n * K)
        tape.append((fpre, y, cache, r))
    grads = np.zeros(gnn.N_TRAINABLE)
    gpost = np.zeros((q, ny * nx))
    for fpre, y, cache, r in reversed(tape):
        gpost = gpost + 2.0 * r.reshape(q, -1) / (n * K)
        dy, dfd = collide_adjoint_channel(fpre, y, tau, p, gx, gpost)
        g, dfn = gnn.backward(dy, cache, p)
        grads += gnn.pack_grads(g)
        gpost = stream_pull_walls_adjoint((dfd + dfn).reshape(q, ny, nx)).reshape(q, -1)
    return loss, grads, gpost.reshape(q, ny, nx)
