"""FP64 oracle for the GNN-enhanced collision and its hand-derived backward.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper passages followed:
  * Sec. 2.2 -- the network: a feature-extraction module over the
    pre-collision populations and the macroscopic variables, a message-passing
    mechanism between neighbouring nodes, and a head predicting the
    tau adjustment and the population corrections.
  * Sec. 2.3.1, Fig. 2 -- inputs [f_0..f_8, rho, u_x, u_y] concatenated; the
    tau head is a sigmoid scaled to the range [0.5, 1.5]; the second head
    predicts the corrections Delta f_i directly.
  * Eq. 3 -- f_i^* = f_i - (f_i - f_i^eq)/(tau tau_adj) + Delta f_i.

Readings where the paper gives no formula:
  * Widths: encoder 12-64-64 (two Linear layers, each followed by GELU),
    two message-passing rounds with separate weights, edge MLP 130->64 and
    node MLP 128->64 (each one Linear + GELU), head 64->10 (linear).
  * Message passing over the 8 lattice neighbours j = i + e_k (k = 1..8,
    periodic): m_ik = GELU(W_e [h_i; h_j; e_k] + b_e), a_i = sum_k m_ik,
    residual node update h_i <- h_i + GELU(W_n [h_i; a_i] + b_n).
  * GELU is the tanh form 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))).
  * tau_adj = 0.5 + sigmoid(y_0); Delta f_i = s_df * y_{1+i}.
  * Inputs are normalised x_hat = (x - mu) / sigma with a fixed (mu, sigma)
    carried with the parameters; s_df likewise.
  * The channel's graph (Sec. 3.1 flow; ``forward(walls=True)``): periodic
    in x, no neighbour beyond the walls past the first and last rows, so
    those messages are left out of the sum and, in ``backward``, pass no
    gradient; with a body force the velocity feature is (j + F/2) / rho.
  * Both sides evaluate the same network: every weight MATRIX is rounded to
    bfloat16 (round to nearest even) before use, biases and (mu, sigma, s_df)
    are used as the float32 values given.  The oracle then computes in FP64.

Variants (the last fixed value, a small integer of flags):
  * 1, MLP-only: the paper's SimpleLBMGNN of Fig. 2 -- the two encoder
    layers use ReLU ("Linear + ReLU" in Fig. 2), there is no message passing,
    and the head reads h0.
  * 2, conservative correction: Delta f is projected onto the populations
    that carry no mass and no momentum (Euclidean projection orthogonal to
    1, e_x, e_y; for D2Q9 these are orthogonal with norms 9, 6, 6), so that
    Eq. 3 conserves mass and momentum like Eq. 1.
  * 4, fixed relaxation time: tau_adj = 1 in Eq. 3 whatever y_0 is (the
    head's first output is unused; dL/dy_0 = 0), so the network corrects
    through Delta f alone and Eq. 3 keeps the BGK relaxation time.

Flat parameter vector (float32, 38,922 trainable values, in this order):
  enc1.W[64,12] enc1.b[64] enc2.W[64,64] enc2.b[64]
  {edge.W[64,130] edge.b[64] node.W[64,128] node.b[64]} for round 1, round 2
  head.W[10,64] head.b[10]
followed by 26 fixed values: mu[12], sigma[12], s_df, variant.
"""
import numpy as np

from . import lbm

HID = 64
NFEAT = 12
NOUT = 10
ROUNDS = 2

SHAPES = [("enc1.W", (HID, NFEAT)), ("enc1.b", (HID,)),
          ("enc2.W", (HID, HID)), ("enc2.b", (HID,))]
for _r in range(ROUNDS):
    SHAPES += [(f"r{_r}.edge.W", (HID, 2 * HID + 2)), (f"r{_r}.edge.b", (HID,)),
               (f"r{_r}.node.W", (HID, 2 * HID)), (f"r{_r}.node.b", (HID,))]
SHAPES += [("head.W", (NOUT, HID)), ("head.b", (NOUT,))]
N_TRAINABLE = sum(int(np.prod(s)) for _, s in SHAPES)
N_FIXED = 2 * NFEAT + 2
MLP_ONLY = 1
CONSERVATIVE = 2
FIXED_TAU = 4
N_TOTAL = N_TRAINABLE + N_FIXED


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even), as float32."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(a32.shape)


def unpack(theta, round_weights=True):
    """Split the flat float32 vector into named FP64 arrays.

    With round_weights, every 2-D weight is first rounded to bfloat16 (the
    shared effective network, see the module docstring)."""
    theta = np.asarray(theta, dtype=np.float32)
    assert theta.shape == (N_TOTAL,), theta.shape
    p = {}
    o = 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        v = theta[o:o + n].reshape(shape)
        if round_weights and len(shape) == 2:
            v = bf16_round(v)
        p[name] = v.astype(np.float64)
        o += n
    p["mu"] = theta[o:o + NFEAT].astype(np.float64)
    p["sigma"] = theta[o + NFEAT:o + 2 * NFEAT].astype(np.float64)
    p["s_df"] = float(theta[o + 2 * NFEAT])
    p["variant"] = int(round(float(theta[o + 2 * NFEAT + 1])))
    return p


def pack_grads(g):
    """Concatenate gradients in the flat trainable order (FP64)."""
    return np.concatenate([np.asarray(g[name], np.float64).ravel() for name, _ in SHAPES])


# --- activations ---------------------------------------------------------------
_C = np.sqrt(2.0 / np.pi)
_A = 0.044715


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(_C * (z + _A * z ** 3)))


def gelu_grad(z):
    t = np.tanh(_C * (z + _A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * _C * (1.0 + 3.0 * _A * z * z)


def relu(z):
    return np.maximum(z, 0.0)


def relu_grad(z):
    return (np.asarray(z) > 0.0).astype(np.float64)


def sigmoid(z):
    """Logistic function, written as 1/2 (1 + tanh(z/2)) (no overflow)."""
    return 0.5 * (1.0 + np.tanh(0.5 * np.asarray(z, np.float64)))


# --- graph of the lattice --------------------------------------------------------
def neighbours(nx, ny):
    """nbr[n, k] = index of node (x + e_kx, y + e_ky) (periodic), n = y*nx + x."""
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    nbr = np.empty((ny * nx, lbm.Q), dtype=np.int64)
    for k in range(lbm.Q):
        xx = (x + lbm.E[k, 0]) % nx
        yy = (y + lbm.E[k, 1]) % ny
        nbr[:, k] = (yy * nx + xx).ravel()
    return nbr


# --- forward ---------------------------------------------------------------------
def inside_mask(nx, ny):
    """inside[n, k]: the neighbour x + e_k of node n lies inside a channel with
    walls beyond the first and last rows (periodic in x only)."""
    y = np.repeat(np.arange(ny), nx)
    return np.stack([(y + lbm.E[k, 1] >= 0) & (y + lbm.E[k, 1] < ny) for k in range(lbm.Q)],
                    axis=1)


def features(f_pre, p, force_x=0.0):
    """Fig. 2 input: [f_0..f_8, rho, u_x, u_y] per node, then (x - mu)/sigma.

    f_pre: (9, ny, nx) pre-collision populations.  With a body force (the
    channel of Sec. 3.1, Guo's scheme) u is the force-corrected velocity
    (sum f e + F/2) / rho.  Returns (N, 12) x_hat and the raw (N, 12)
    feature matrix."""
    rho, ux, uy = lbm.moments(f_pre)
    ux = ux + 0.5 * force_x / rho
    q = f_pre.shape[0]
    raw = np.concatenate([np.asarray(f_pre, np.float64).reshape(q, -1).T,
                          rho.reshape(-1, 1), ux.reshape(-1, 1), uy.reshape(-1, 1)], axis=1)
    return (raw - p["mu"]) / p["sigma"], raw


def forward(f_pre, p, walls=False, force_x=0.0):
    """Network output y (N, 10) for pre-collision populations f_pre (9, ny, nx).

    The edge MLP is applied per edge to the full 130-wide concatenation
    [h_i; h_j; e_k] (brute force, no algebraic split).  walls: the channel's
    graph (periodic in x, no neighbour across the walls beyond the first and
    last rows: such messages are left out of the sum); force_x: the body
    force of the channel (forced velocity in the features).  Returns
    (y, cache)."""
    _, ny, nx = f_pre.shape
    nbr = neighbours(nx, ny)
    keep = inside_mask(nx, ny) if walls else np.ones((nx * ny, lbm.Q), bool)
    xh, raw = features(f_pre, p, force_x)
    act = relu if p["variant"] & MLP_ONLY else gelu
    z1 = xh @ p["enc1.W"].T + p["enc1.b"]
    g1 = act(z1)
    z2 = g1 @ p["enc2.W"].T + p["enc2.b"]
    h = act(z2)
    cache = {"nbr": nbr, "xh": xh, "raw": raw, "z1": z1, "g1": g1, "z2": z2,
             "h": [h], "edge_in": [], "ze": [], "a": [], "zn": [], "walls": walls,
             "keep": keep}
    for r in range(0 if p["variant"] & MLP_ONLY else ROUNDS):
        We, be = p[f"r{r}.edge.W"], p[f"r{r}.edge.b"]
        Wn, bn = p[f"r{r}.node.W"], p[f"r{r}.node.b"]
        a = np.zeros_like(h)
        ins, zes = [], []
        for k in range(1, lbm.Q):
            ek = np.broadcast_to(lbm.E[k].astype(np.float64), (h.shape[0], 2))
            inp = np.concatenate([h, h[nbr[:, k]], ek], axis=1)   # (N, 130)
            ze = inp @ We.T + be
            a = a + gelu(ze) * keep[:, k:k + 1]
            ins.append(inp)
            zes.append(ze)
        zn = np.concatenate([h, a], axis=1) @ Wn.T + bn
        h = h + gelu(zn)
        cache["edge_in"].append(ins)
        cache["ze"].append(zes)
        cache["a"].append(a)
        cache["zn"].append(zn)
        cache["h"].append(h)
    y = h @ p["head.W"].T + p["head.b"]
    return y, cache


def forward_split(f_pre, p):
    """Same network with the edge MLP split algebraically,
    W_e [h_i; h_j; e_k] = W_a h_i + W_b h_j + W_c e_k.  Used only to pin the
    brute-force form (they must agree to FP64 round-off)."""
    _, ny, nx = f_pre.shape
    nbr = neighbours(nx, ny)
    xh, _ = features(f_pre, p)
    h = gelu(gelu(xh @ p["enc1.W"].T + p["enc1.b"]) @ p["enc2.W"].T + p["enc2.b"])
    for r in range(ROUNDS):
        We, be = p[f"r{r}.edge.W"], p[f"r{r}.edge.b"]
        Wa, Wb, Wc = We[:, :HID], We[:, HID:2 * HID], We[:, 2 * HID:]
        Wn, bn = p[f"r{r}.node.W"], p[f"r{r}.node.b"]
        A = h @ Wa.T
        B = h @ Wb.T
        a = np.zeros_like(h)
        for k in range(1, lbm.Q):
            ck = Wc @ lbm.E[k].astype(np.float64) + be
            a = a + gelu(A + B[nbr[:, k]] + ck)
        h = h + gelu(h @ Wn[:, :HID].T + a @ Wn[:, HID:].T + bn)
    return h @ p["head.W"].T + p["head.b"]


def conserve(df):
    """Projection of corrections (9, N) orthogonal to 1, e_x, e_y:
    df - sum(df)/9 - e_x sum(e_x df)/6 - e_y sum(e_y df)/6."""
    ex = lbm.E[:, 0].astype(np.float64)[:, None]
    ey = lbm.E[:, 1].astype(np.float64)[:, None]
    return (df - df.sum(axis=0) / 9.0 - ex * (ex * df).sum(axis=0) / 6.0
            - ey * (ey * df).sum(axis=0) / 6.0)


def heads(y, p):
    """Sec. 2.3.1: tau_adj = 0.5 + sigmoid(y_0) in (0.5, 1.5) (1 with the
    fixed-tau variant); Delta f_i = s_df * y_{1+i} (projected with the
    conservative variant).  Returns tau_adj (N,), df (9, N)."""
    df = p["s_df"] * y[:, 1:].T
    if p["variant"] & CONSERVATIVE:
        df = conserve(df)
    if p["variant"] & FIXED_TAU:
        return np.ones(y.shape[0]), df
    return 0.5 + sigmoid(y[:, 0]), df


def gnn_collide(f_pre, y, tau, p):
    """Eq. 3: f* = f - (f - f^eq)/(tau tau_adj) + Delta f, on (9, ny, nx)."""
    q, ny, nx = f_pre.shape
    rho, ux, uy = lbm.moments(f_pre)
    feq = lbm.equilibrium(rho, ux, uy).reshape(q, -1)
    f = np.asarray(f_pre, np.float64).reshape(q, -1)
    tau_adj, df = heads(y, p)
    return (f - (f - feq) / (tau * tau_adj) + df).reshape(q, ny, nx)


def gnn_step(f_post, theta, tau):
    """One GNN-LBM step on the stored post-collision state (Fig. 1 'Use GNN?'
    = yes): pull-stream, network on the pre-collision state, Eq. 3."""
    p = unpack(theta)
    f_pre = lbm.stream_pull(f_post)
    y, _ = forward(f_pre, p)
    return gnn_collide(f_pre, y, tau, p)


# --- backward --------------------------------------------------------------------
def backward(dy, cache, p):
    """Reverse mode of ``forward`` given dL/dy (N, 10).

    Returns (grads, d_f_pre): grads maps every trainable name to dL/d(param)
    in FP64 (w.r.t. the effective, already rounded values); d_f_pre is
    dL/d f_pre (9, N) through the features (f_i, rho, u).  On the channel's
    graph (forward with walls) an edge that the forward left out of the sum
    passes no gradient; with a body force the velocity feature is
    (j + F/2)/rho, whose derivative w.r.t. f_i is (e_i - u)/rho with that u
    (cache "raw" holds it)."""
    keep = cache.get("keep")
    g = {}
    nbr = cache["nbr"]
    h = cache["h"][-1]
    g["head.W"] = dy.T @ h
    g["head.b"] = dy.sum(axis=0)
    dh = dy @ p["head.W"]
    for r in reversed(range(0 if p["variant"] & MLP_ONLY else ROUNDS)):
        We = p[f"r{r}.edge.W"]
        Wn = p[f"r{r}.node.W"]
        h_in = cache["h"][r]
        a = cache["a"][r]
        dzn = dh * gelu_grad(cache["zn"][r])
        g[f"r{r}.node.W"] = dzn.T @ np.concatenate([h_in, a], axis=1)
        g[f"r{r}.node.b"] = dzn.sum(axis=0)
        dcat = dzn @ Wn
        dh_in = dh + dcat[:, :HID]
        da = dcat[:, HID:]
        gWe = np.zeros_like(We)
        gbe = np.zeros(HID)
        for kk, k in enumerate(range(1, lbm.Q)):
            dze = da * gelu_grad(cache["ze"][r][kk])
            if keep is not None:
                dze = dze * keep[:, k:k + 1]
            gWe += dze.T @ cache["edge_in"][r][kk]
            gbe += dze.sum(axis=0)
            dinp = dze @ We
            dh_in += dinp[:, :HID]
            np.add.at(dh_in, nbr[:, k], dinp[:, HID:2 * HID])
        g[f"r{r}.edge.W"] = gWe
        g[f"r{r}.edge.b"] = gbe
        dh = dh_in
    if p["variant"] & MLP_ONLY:
        for r in range(ROUNDS):
            for name in ("edge.W", "edge.b", "node.W", "node.b"):
                g[f"r{r}.{name}"] = np.zeros_like(p[f"r{r}.{name}"])
    dact = relu_grad if p["variant"] & MLP_ONLY else gelu_grad
    dz2 = dh * dact(cache["z2"])
    g["enc2.W"] = dz2.T @ cache["g1"]
    g["enc2.b"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["enc2.W"]) * dact(cache["z1"])
    g["enc1.W"] = dz1.T @ cache["xh"]
    g["enc1.b"] = dz1.sum(axis=0)
    dx = (dz1 @ p["enc1.W"]) / p["sigma"]          # d/d raw features (N, 12)
    raw = cache["raw"]
    rho, ux, uy = raw[:, 9], raw[:, 10], raw[:, 11]
    df = dx[:, :9].T.copy()                          # direct f_i inputs
    for i in range(lbm.Q):                           # through rho and u = j/rho
        df[i] += dx[:, 9] + (dx[:, 10] * (lbm.E[i, 0] - ux)
                             + dx[:, 11] * (lbm.E[i, 1] - uy)) / rho
    return g, df


def collide_loss(f_pre, y, tau, target, p, node_weight=None):
    """Eq. 3 followed by Eq. 4 (mean over nodes x 9 of the squared error).

    tau may be a scalar or a per-node array (N,).  node_weight (N,), optional:
    each node's squared error multiplied by it (the per-instance weights of
    the library's weighted training step; None is Eq. 4).  Returns (loss,
    dL/dy (N,10), f_pred (9, N))."""
    q = f_pre.shape[0]
    rho, ux, uy = lbm.moments(f_pre)
    feq = lbm.equilibrium(rho, ux, uy).reshape(q, -1)
    f = np.asarray(f_pre, np.float64).reshape(q, -1)
    t = np.asarray(target, np.float64).reshape(q, -1)
    tau_adj, df = heads(y, p)
    teff = tau * tau_adj
    f_pred = f - (f - feq) / teff + df
    n = f.size
    r = f_pred - t
    wn = 1.0 if node_weight is None else np.asarray(node_weight, np.float64)[None, :]
    loss = float(np.sum(wn * r * r) / n)
    dfs = 2.0 * wn * r / n                           # dL/d f*
    dy = np.zeros_like(y)
    # Delta f = s_df P y_1..9 with P symmetric (P = I without the variant)
    dy[:, 1:] = (p["s_df"] * (conserve(dfs) if p["variant"] & CONSERVATIVE else dfs)).T
    dtau_adj = np.sum(dfs * (f - feq), axis=0) * tau / (teff * teff)
    s = sigmoid(y[:, 0])
    dy[:, 0] = 0.0 if p["variant"] & FIXED_TAU else dtau_adj * s * (1.0 - s)
    return loss, dy, f_pred
