"""FP64 oracle for the training side: data generation from a refined lattice,
restriction to the coarse lattice, and the AdamW update.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
  * Sec. 2.4 -- supervised training on pairs generated by high-resolution
    standard LBM runs; the loss is Eq. 4 (``oracle.gnn.collide_loss``).

Readings where the paper is silent:
  * "High resolution" = an m-times refined lattice (m = 4 by default) under
    acoustic scaling: the same lattice velocity u0, k_f = k_c / m,
    tau_f = 1/2 + m (tau_c - 1/2), and m fine steps per coarse step.
  * Coarse node (I, J) coincides with fine node (m I, m J).
  * Restriction (Dupuis-Chopard rescaling): rho and u are injected from the
    fine node; the non-equilibrium part of the fine PRE-collision state is
    recovered from the stored post-collision one,
        f_neq_f = (f*_f - f^eq) / (1 - 1/tau_f),
    rescaled to the coarse lattice, f_neq_c = m (tau_c / tau_f) f_neq_f, and
    the coarse post-collision state is f*_c = f^eq + (1 - 1/tau_c) f_neq_c.
  * Channel (forced) data: an odd factor m (3) so that fine and coarse nodes
    coincide with the walls halfway beyond the outer rows, the force scaled
    as F_f = F_c / m, and the restriction of ``restrict_forced``, which
    separates the force part of the non-equilibrium populations from the
    gradient part and works from the pre-collision state.
  * A training pair is (restricted state at coarse step n, at step n+1); the
    prediction is one GNN-LBM coarse step on the first element.
  * K-step rollout loss (``rollout_loss``; an option beyond Eq. 4, which is
    its K = 1 case): the mean of Eq. 4 over K consecutive GNN-LBM steps from
    the restricted state against the restricted refined run, differentiated
    through the dynamics (adjoints of Eq. 3 and of streaming).
  * The optimiser (unnamed in the paper) is AdamW with decoupled weight decay
    (Loshchilov & Hutter): beta = (0.9, 0.999), eps = 1e-8.
"""
import numpy as np

from . import lbm


def fine_tau(tau_c, m):
    """tau of the m-times refined lattice that keeps the physical viscosity."""
    return 0.5 + m * (tau_c - 0.5)


def restrict(f_fine, m, tau_f, tau_c):
    """Restrict a fine post-collision state (9, m ny, m nx) to the coarse one."""
    sub = np.asarray(f_fine, np.float64)[:, ::m, ::m]
    rho, ux, uy = lbm.moments(sub)
    feq = lbm.equilibrium(rho, ux, uy)
    fneq_f = (sub - feq) / (1.0 - 1.0 / tau_f)
    fneq_c = m * (tau_c / tau_f) * fneq_f
    return feq + (1.0 - 1.0 / tau_c) * fneq_c


def restrict_forced(f_pre_fine, m, tau_f, tau_c, gx_f):
    """Restrict a fine channel state, given PRE-collision (9, m ny, m nx),
    to the coarse post-collision state at the same time (readings for a
    forced flow, Sec. 2.4 with Sec. 3.1):
      * m odd; coarse node (I, J) coincides with fine node (m I + (m-1)/2,
        m J + (m-1)/2), so both lattices put their walls halfway beyond the
        outer rows;
      * the force per unit volume scales as F_f = F_c / m (same lattice
        velocity with nu_f = m nu_c on an m-times wider channel);
      * the non-equilibrium part of the pre-collision state splits into a
        gradient part G = -tau D f^eq, which scales to the coarse lattice by
        m tau_c / tau_f, and a force part P = (tau - 1/2) w_i [3 (e_i - u) +
        9 (e_i . u) e_i] . F, which is the same in both lattices' units;
      * the coarse post-collision state is
            f*_c = f^eq + (1 - 1/tau_c) m (tau_c / tau_f) G + P.
    The pre-collision state is used because the post-collision one holds
    (1 - 1/tau_f) G, whose inversion fails at tau_f = 1."""
    from . import channel
    assert m % 2 == 1, "co-located nodes need an odd refinement factor"
    o = (m - 1) // 2
    sub = np.asarray(f_pre_fine, np.float64)[:, o::m, o::m]
    rho, ux, uy = channel.moments_forced(sub, gx_f)
    feq = lbm.equilibrium(rho, ux, uy)
    pf = (tau_f - 0.5) * channel.guo_term(ux, uy, gx_f)
    g = sub - feq - pf
    return feq + (1.0 - 1.0 / tau_c) * m * (tau_c / tau_f) * g + pf


def channel_pair(ny_c, nx_c, tau_c, gx_c, n_steps, m=3, f0_fine=None):
    """One training pair on an ny_c x nx_c coarse channel (force gx_c): the
    fine channel (m ny_c x m nx_c, tau_f, F_c / m) runs from f0_fine (rest
    when None) for m n_steps - 1 steps; its pull with the walls is the
    pre-collision state at coarse step n, restricted to f_in; m more fine
    steps give the target.  Returns (f_in, f_target)."""
    from . import channel
    tau_f = fine_tau(tau_c, m)
    gx_f = gx_c / m
    f = (lbm.equilibrium(np.ones((m * ny_c, m * nx_c)), np.zeros((m * ny_c, m * nx_c)),
                         np.zeros((m * ny_c, m * nx_c)))
         if f0_fine is None else np.asarray(f0_fine, np.float64))
    f = channel.channel_run(f, tau_f, gx_f, m * n_steps - 1)
    f_in = restrict_forced(channel.stream_pull_walls(f), m, tau_f, tau_c, gx_f)
    f = channel.channel_run(f, tau_f, gx_f, m)
    return f_in, restrict_forced(channel.stream_pull_walls(f), m, tau_f, tau_c, gx_f)


def tgv_pair(n_c, u0, k_mult, tau_c, n_steps, m=4):
    """One training pair on an n_c x n_c coarse TGV with wavenumber
    k = k_mult * 2 pi / n_c: the fine lattice (m n_c)^2 is run m*n_steps and
    then m more steps; both ends are restricted.  Returns (f_in, f_target)."""
    n_f = m * n_c
    k_f = k_mult * 2.0 * np.pi / n_f
    tau_f = fine_tau(tau_c, m)
    f = lbm.tgv_init(n_f, n_f, 1.0, u0, k_f, k_f)
    f = lbm.bgk_run(f, tau_f, m * n_steps)
    f_in = restrict(f, m, tau_f, tau_c)
    f = lbm.bgk_run(f, tau_f, m)
    return f_in, restrict(f, m, tau_f, tau_c)


def collide_adjoint(f_pre, y, tau, p, g):
    """Reverse mode of Eq. 3 given g = dL/df* (9, N): returns dL/dy (N, 10)
    and the part of dL/df_pre (9, N) that passes through the explicit f and
    f^eq(rho(f), u(f)) of Eq. 3 (the network's own dependence on f_pre is
    ``gnn.backward``'s d_f_pre).  With t = tau tau_adj:
      d f*_i / d f_j = delta_ij (1 - 1/t) + (1/t) d f^eq_i / d f_j,
      d f^eq_i / d f_j = f^eq_i / rho
                         + w_i [3 e_i + 9 (e_i . u) e_i - 3 u] . (e_j - u),
    the second line from Eq. 2 with rho = sum f, u = sum f e / rho."""
    from . import gnn
    q = lbm.Q
    f = np.asarray(f_pre, np.float64).reshape(q, -1)
    rho, ux, uy = lbm.moments(f)
    feq = lbm.equilibrium(rho, ux, uy)
    g = np.asarray(g, np.float64).reshape(q, -1)
    tau_adj, _ = gnn.heads(y, p)
    t = tau * tau_adj
    dy = np.zeros_like(y)
    dy[:, 1:] = (p["s_df"] * (gnn.conserve(g) if p["variant"] & gnn.CONSERVATIVE else g)).T
    s = gnn.sigmoid(y[:, 0])
    dy[:, 0] = (0.0 if p["variant"] & gnn.FIXED_TAU
                else np.sum(g * (f - feq), axis=0) / (t * t) * tau * s * (1.0 - s))
    a = np.sum(g * feq, axis=0) / rho                      # sum_i g_i f^eq_i / rho
    vx = np.zeros_like(rho)
    vy = np.zeros_like(rho)
    for i in range(q):
        ex, ey = lbm.E[i]
        eu = ex * ux + ey * uy
        vx += g[i] * lbm.W[i] * (3.0 * ex + 9.0 * eu * ex - 3.0 * ux)
        vy += g[i] * lbm.W[i] * (3.0 * ey + 9.0 * eu * ey - 3.0 * uy)
    df = np.empty_like(f)
    for j in range(q):
        ex, ey = lbm.E[j]
        df[j] = g[j] * (1.0 - 1.0 / t) + (a + vx * (ex - ux) + vy * (ey - uy)) / t
    return dy, df


def rollout_loss(f0, targets, theta, tau):
    """K-step rollout loss (this library's training option; the paper's Eq. 4
    is the one-step case K = 1): K GNN-LBM steps (stream, network, Eq. 3)
    from the stored state f0 (9, ny, nx), and the mean over the K steps of
    Eq. 4 against targets[k] (the refined run's restricted state after k + 1
    coarse steps).  theta: a parameter vector, or the dict of
    ``gnn.unpack`` (its values used as given).  Returns (loss, packed
    dL/dtheta (38,922), dL/df0), the
    gradient by reverse mode through every step: the adjoint of Eq. 3
    (``collide_adjoint``), the network's backward (``gnn.backward``, with its
    d_f_pre) and the adjoint of streaming (``lbm.stream_pull_adjoint``)."""
    from . import gnn
    p = theta if isinstance(theta, dict) else gnn.unpack(theta)
    K = len(targets)
    f = np.asarray(f0, np.float64)
    q, ny, nx = f.shape
    n = f.size
    tape = []
    loss = 0.0
    for k in range(K):
        fpre = lbm.stream_pull(f)
        y, cache = gnn.forward(fpre, p)
        f = gnn.gnn_collide(fpre, y, tau, p)
        r = f - np.asarray(targets[k], np.float64)
        loss += float(np.sum(r * r)) / (n * K)
        tape.append((fpre, y, cache, r))
    grads = np.zeros(gnn.N_TRAINABLE)
    gpost = np.zeros((q, ny * nx))
    for fpre, y, cache, r in reversed(tape):
        gpost = gpost + 2.0 * r.reshape(q, -1) / (n * K)
        dy, dfd = collide_adjoint(fpre, y, tau, p, gpost)
        g, dfn = gnn.backward(dy, cache, p)
        grads += gnn.pack_grads(g)
        gpost = lbm.stream_pull_adjoint((dfd + dfn).reshape(q, ny, nx)).reshape(q, -1)
    return loss, grads, gpost.reshape(q, ny, nx)


def pair_weights(f_in, f_target, taus, wmax=1.0e4):
    """Per-instance loss weights of a stack of training pairs (this
    library's training option): D_b = mean over nodes x 9 of (BGK step of
    f_in[b]) - f_target[b])^2 (Eq. 1-2), w_b = mean(D) / D_b capped at wmax.
    f_in, f_target: lists of (9, ny, nx) states; taus: per instance.
    Returns (D, w)."""
    d = np.array([np.mean((lbm.bgk_step(np.asarray(a, np.float64), t)
                           - np.asarray(b, np.float64)) ** 2)
                  for a, b, t in zip(f_in, f_target, taus)])
    mean = d.mean()
    w = np.where(d * wmax > mean, mean / np.where(d > 0, d, 1.0), wmax)
    return d, w


def adamw_step(theta, grad, m, v, t, lr, wd, beta1=0.9, beta2=0.999, eps=1e-8):
    """One AdamW update at step t (1-based).  Returns (theta, m, v)."""
    theta = np.asarray(theta, np.float64) * (1.0 - lr * wd)
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
