"""Training of the GNN-enhanced collision on data the library generates
(paper Sec. 2.4), driven through the C ABI.

Every arithmetic step runs in liblbmgnn.so: the refined-lattice Taylor-Green
runs (lbm_init_tgv_batch, lbm_step_bgk with per-lattice tau), the restriction
to the coarse lattice (lbm_restrict), and the fused training step
(gnn_train_step: stream, network forward, Eq. 3, Eq. 4, backward, AdamW,
repack).  This module only allocates device buffers, draws the per-instance
flow parameters (seeded) and sequences the calls.

Data (readings of Sec. 2.4 listed with the restriction in include/lbmgnn.h):
instances are periodic TGVs on an n x n coarse lattice with k = k_mult 2 pi/n,
k_mult in {1, 2, 4}, u0 ~ U[0.01, 0.08], Re ~ U[100, 5000] with Re = u0 n / nu.
The refined lattice is m n (m = 4) with the same u0, k_f = k/m and
tau_f = 1/2 + m (tau - 1/2); m fine steps make one coarse step.  A training
pair is (restricted state at coarse step t, restricted state at t + 1).
The refined runs start from the pressure-consistent TGV density by default,
so that the pairs carry no start-up acoustic transient.
"""
import numpy as np

from . import inputs
from . import lib as L


class PairStream:
    """Batches of training pairs from `batch` refined-lattice TGV runs.

    Each episode draws fresh instances, initialises the fine lattices at
    equilibrium and yields `episode` consecutive coarse pairs."""

    def __init__(self, device, n=256, batch=64, m=4, episode=32, seed=0,
                 pressure_consistent=True, instances=None):
        import torch
        self.dev = device
        # keyword arguments of inputs.training_instances (u0_range, re_range,
        # log_re): the distribution of the TGV instances
        self.instance_kw = dict(instances or {})
        self.n, self.batch, self.m, self.episode = n, batch, m, episode
        self.rng_seed = seed
        self.draw = 0
        nf = m * n
        self.fine = L.shape(nf, nf, batch)
        self.coarse = L.shape(n, n, batch)
        self.ff = [torch.empty(9 * batch * nf * nf, device=device) for _ in range(2)]
        self.fc = [torch.empty(9 * batch * n * n, device=device) for _ in range(2)]
        self.tau_c = torch.empty(batch, device=device)
        self.tau_f = torch.empty(batch, device=device)
        self.prm = torch.empty(batch * 4, dtype=torch.float64, device=device)
        self.pc = pressure_consistent
        self.t = episode  # forces a new episode on the first call

    def _new_episode(self):
        import torch
        inst = inputs.training_instances(self.batch, self.rng_seed * 100003 + self.draw, self.n,
                                         **self.instance_kw)
        self.draw += 1
        nf = self.m * self.n
        prm = np.zeros((self.batch, 4))
        tc = np.zeros(self.batch, np.float32)
        for b, d in enumerate(inst):
            kf = d["k_mult"] * 2 * np.pi / nf
            prm[b] = (1.0, d["u0"], kf, kf)
            tc[b] = 0.5 + 3.0 * d["nu"]
        tf = (0.5 + self.m * (tc.astype(np.float64) - 0.5)).astype(np.float32)
        self.instances = inst
        self.prm.copy_(torch.from_numpy(prm.reshape(-1)))
        self.tau_c.copy_(torch.from_numpy(tc))
        self.tau_f.copy_(torch.from_numpy(tf))
        L.lbm_init_tgv_batch(self.ff[0], self.fine, self.prm, self.pc)
        L.lbm_restrict(self.ff[0], self.fine, self.fc[0], self.coarse, self.m, 0.0, self.tau_f,
                       0.0, self.tau_c)
        self.t = 0

    def next(self):
        """Advance one coarse step; returns (f_in, f_target, tau_c) device
        tensors valid until the next call."""
        if self.t >= self.episode:
            self._new_episode()
        # m fine steps: ff[0] -> ff[1] -> ff[0] ... ending in ff[0]
        for _ in range(self.m):
            L.lbm_step_bgk(self.ff[0], self.ff[1], None, self.fine, 1.0, taus=self.tau_f, nsteps=1)
            self.ff.reverse()
        src, dst = self.fc[0], self.fc[1]
        L.lbm_restrict(self.ff[0], self.fine, dst, self.coarse, self.m, 0.0, self.tau_f, 0.0,
                       self.tau_c)
        self.fc.reverse()
        self.t += 1
        return src, dst, self.tau_c


class Trainer:
    """AdamW training of the network on a PairStream (fused C ABI step).

    weighting: "eq4" (the paper's loss) or "relative" (each training instance
    weighted by mean(D) / D_b, D_b its one-step BGK residual: lbm_pair_weights
    and gnn_train_step_weighted)."""

    def __init__(self, device, theta=None, lr=1e-3, wd=1e-2, seed=0, weighting="eq4",
                 **stream_kw):
        import torch
        self.data = PairStream(device, seed=seed, **stream_kw)
        theta = inputs.xavier_params(seed) if theta is None else theta
        self.params = torch.from_numpy(np.asarray(theta, np.float32)).to(device)
        self.packed = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=device)
        L.gnn_pack(self.params, self.packed)
        self.m = torch.zeros(L.gnn_trainable_count(), device=device)
        self.v = torch.zeros_like(self.m)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.ws = torch.empty(L.gnn_train_workspace_bytes(self.data.coarse), dtype=torch.uint8,
                              device=device)
        self.lr, self.wd = lr, wd
        self.step_count = 0
        if weighting not in ("eq4", "relative"):
            raise ValueError(f"unknown weighting {weighting!r}")
        self.weighting = weighting
        if weighting == "relative":
            nb = self.data.coarse.nb
            self.lat_w = torch.ones(nb, device=device)
            self.pw_ws = torch.empty(L.lbm_pair_weights_workspace_bytes(self.data.coarse),
                                     dtype=torch.uint8, device=device)

    def step(self):
        f_in, f_tg, tau_c = self.data.next()
        self.step_count += 1
        if self.weighting == "relative":
            L.lbm_pair_weights(f_in, f_tg, self.data.coarse, 1.0, tau_c, self.lat_w, self.pw_ws)
            L.gnn_train_step_weighted(f_in, f_tg, self.data.coarse, 1.0, tau_c, self.lat_w,
                                      self.params, self.packed, self.m, self.v, self.step_count,
                                      self.lr, self.wd, self.loss, None, self.ws)
            return
        L.gnn_train_step(f_in, f_tg, self.data.coarse, 1.0, tau_c, self.params, self.packed,
                         self.m, self.v, self.step_count, self.lr, self.wd, self.loss, None,
                         self.ws)

    def theta(self):
        return self.params.cpu().numpy().copy()


class RolloutStream:
    """K-step training windows from the refined-lattice TGV runs of a
    PairStream: the restricted state at coarse step t and the K restricted
    states after it, targets contiguous ([K] x 9 planes), for
    gnn_train_step_rollout.  `episode` windows per episode of refined runs; a
    window never spans two episodes; consecutive windows of an episode
    overlap (a sliding window)."""

    def __init__(self, device, K=4, episode=32, **pair_kw):
        import torch
        self.K = K
        # episode + K - 1 pairs give episode + K states: `episode` windows
        self.pairs = PairStream(device, episode=episode + K - 1, **pair_kw)
        self.coarse = self.pairs.coarse
        n = 9 * self.coarse.nx * self.coarse.ny * self.coarse.nb
        self.ring = [torch.empty(n, device=device) for _ in range(K + 1)]
        self.f_in = torch.empty(n, device=device)
        self.targets = torch.empty(K * n, device=device)
        self.count = 0

    def next(self):
        """Returns (f_in, targets, tau_c) device tensors valid until the next
        call."""
        K = self.K
        while True:
            src, dst, taus = self.pairs.next()
            if self.pairs.t == 1:                 # a new episode began
                self.ring[0].copy_(src)
                self.count = 1
            self.ring[self.count % (K + 1)].copy_(dst)
            self.count += 1
            if self.count >= K + 1:
                break
        first = self.count - (K + 1)
        n = self.f_in.numel()
        self.f_in.copy_(self.ring[first % (K + 1)])
        for k in range(K):
            self.targets[k * n:(k + 1) * n].copy_(self.ring[(first + 1 + k) % (K + 1)])
        return self.f_in, self.targets, taus


class RolloutTrainer:
    """AdamW training of the network on K-step windows (RolloutStream) with
    the rollout loss of gnn_train_step_rollout (the mean of Eq. 4 over K
    GNN-LBM steps, differentiated through the dynamics)."""

    def __init__(self, device, K=4, theta=None, lr=1e-3, wd=1e-2, seed=0, **stream_kw):
        import torch
        self.data = RolloutStream(device, K=K, seed=seed, **stream_kw)
        self.K = K
        theta = inputs.xavier_params(seed) if theta is None else theta
        self.params = torch.from_numpy(np.asarray(theta, np.float32)).to(device)
        self.packed = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=device)
        L.gnn_pack(self.params, self.packed)
        self.m = torch.zeros(L.gnn_trainable_count(), device=device)
        self.v = torch.zeros_like(self.m)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.ws = torch.empty(L.gnn_rollout_workspace_bytes(self.data.coarse, K),
                              dtype=torch.uint8, device=device)
        self.lr, self.wd = lr, wd
        self.step_count = 0

    def step(self):
        f_in, targets, taus = self.data.next()
        self.step_count += 1
        L.gnn_train_step_rollout(f_in, targets, self.K, self.data.coarse, 1.0, taus, self.params,
                                 self.packed, self.m, self.v, self.step_count, self.lr, self.wd,
                                 self.loss, None, self.ws)

    def theta(self):
        return self.params.cpu().numpy().copy()


class Evaluator:
    """Eq. 4 loss of a parameter vector on pairs, without training: stream,
    network forward, Eq. 3 and the loss, all through the C ABI."""

    def __init__(self, device, coarse):
        import torch
        self.s = coarse
        n = coarse.nx * coarse.ny * coarse.nb
        self.f_pre = torch.empty(9 * n, device=device)
        self.saved = torch.empty(L.gnn_saved_bytes(coarse), dtype=torch.uint8, device=device)
        self.y = torch.empty(10 * n, device=device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.ws = torch.empty(L.gnn_loss_workspace_bytes(coarse), dtype=torch.uint8, device=device)
        self.packed = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=device)
        self.dev = device

    def loss_of(self, params, f_in, f_target, taus):
        """params: device FP32 parameter vector; returns the Eq. 4 loss."""
        L.gnn_pack(params, self.packed)
        L.lbm_stream(f_in, self.f_pre, self.s)
        L.gnn_forward(self.f_pre, self.s, self.packed, self.saved, self.y)
        L.gnn_collide_loss(self.f_pre, self.y, f_target, self.s, 1.0, taus, self.packed, self.loss,
                           None, None, self.ws)
        return self.loss.item()


class HeldOutRollout:
    """A held-out Taylor-Green case run three ways through the C ABI: the
    m-times refined BGK reference (m fine steps per coarse step, restricted
    to the coarse lattice when asked), and the coarse lattice advanced from
    the restricted initial state by the BGK step and by the GNN-LBM step
    (parameters `theta`).  Default: the evaluation case of the training
    workload, k = 4 (2 pi / 256), u0 = 0.08, Re = 5000 on 256^2 coarse
    nodes, the refined run started from the pressure-consistent density like
    the training data."""

    def __init__(self, device, theta, n=256, m=4, u0=0.08, k_mult=4, re=5000.0,
                 pressure_consistent=True):
        import torch
        self.dev, self.n, self.m = device, n, m
        nu = u0 * n / re
        self.tau_c = 0.5 + 3.0 * nu
        self.tau_f = 0.5 + m * (self.tau_c - 0.5)
        nf = m * n
        kf = k_mult * 2 * np.pi / nf
        self.fine, self.coarse = L.shape(nf, nf), L.shape(n, n)
        self.ff = [torch.empty(9 * nf * nf, device=device) for _ in range(2)]
        self.fb = [torch.empty(9 * n * n, device=device) for _ in range(2)]
        self.fg = [torch.empty(9 * n * n, device=device) for _ in range(2)]
        self.ref = torch.empty(9 * n * n, device=device)
        L.lbm_init_tgv(self.ff[0], self.fine, 1.0, u0, kf, kf, pressure_consistent)
        L.lbm_restrict(self.ff[0], self.fine, self.fb[0], self.coarse, m, self.tau_f, None,
                       self.tau_c, None)
        self.fg[0].copy_(self.fb[0])
        self.packed = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=device)
        L.gnn_pack(torch.from_numpy(np.asarray(theta, np.float32)).to(device), self.packed)
        self.ws = torch.empty(L.gnn_step_workspace_bytes(self.coarse), dtype=torch.uint8,
                              device=device)
        self.t = 0

    def step(self):
        """One coarse step of all three runs."""
        for _ in range(self.m):
            L.lbm_step_bgk(self.ff[0], self.ff[1], None, self.fine, self.tau_f)
            self.ff.reverse()
        L.lbm_step_bgk(self.fb[0], self.fb[1], None, self.coarse, self.tau_c)
        self.fb.reverse()
        L.lbm_step_gnn(self.fg[0], self.fg[1], self.coarse, self.tau_c, None, self.packed, None,
                       self.ws)
        self.fg.reverse()
        self.t += 1

    def velocities(self):
        """(ux, uy) device planes of the restricted reference, the BGK run
        and the GNN run at the current step."""
        import torch
        L.lbm_restrict(self.ff[0], self.fine, self.ref, self.coarse, self.m, self.tau_f, None,
                       self.tau_c, None)
        out = []
        nn = self.n * self.n
        for f in (self.ref, self.fb[0], self.fg[0]):
            ux, uy = torch.empty(nn, device=self.dev), torch.empty(nn, device=self.dev)
            L.lbm_moments(f, self.coarse, None, ux, uy, None)
            out.append((ux, uy))
        return out


class ChannelPairBank:
    """Training pairs for the channel network (Sec. 2.4 data for the flow of
    Sec. 3.1), generated on the GPU through the C ABI and kept resident.

    `groups` refined channels run from rest (m = 3 times finer, halfway
    bounce-back, Guo forcing; lbm_step_channel with per-lattice tau_f and
    the group's force F_c / m); each group holds `per_group` lattices of one
    force with different viscosities.  Every `snapshot` coarse-step time is a
    pair: lbm_restrict_channel of the fine state one fine step before
    (coarse step n) and m fine steps later (n + 1).  The snapshot times are
    fractions of the group's slowest-mode e-folding time H^2/(pi^2 nu), from
    the start-up transient to the steady state.

    Group draw (seeded): u_ref ~ U[u_range], Re_ref log-uniform in re_range,
    nu_ref = u_ref H / Re_ref, coarse force G = 8 nu_ref u_ref / H^2; lattice
    i of the group takes nu_i = nu_ref s_i with s_i log-uniform in
    [1/spread, spread] (centre-line velocity u_ref / s_i, Re_ref / s_i^2).

    Layout: inputs and targets [9][NB][h][nx] with plane stride NB h nx, NB =
    groups x per_group x len(snapshots); the (group, snapshot) blocks sit in
    a seeded random order, so that batch j (lattices batch*j ..
    batch*(j+1)-1) mixes groups and times.  tau_c and the coarse force per
    lattice: device FP32 [NB]."""

    SNAPSHOTS = (0.02, 0.05, 0.1, 0.2, 0.35, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0, 4.5, 6.0, 8.0)

    def __init__(self, device, h=32, nx=8, m=3, groups=16, per_group=8, snapshots=None,
                 seed=0, u_range=(0.03, 0.07), re_range=(8.0, 250.0), spread=1.5):
        import torch
        if m % 2 == 0:
            raise ValueError("the channel restriction needs an odd refinement factor")
        self.dev, self.h, self.nx, self.m = device, h, nx, m
        self.per_group = per_group
        snaps = tuple(snapshots or self.SNAPSHOTS)
        nblk = groups * len(snaps)
        self.nb = nblk * per_group
        per = h * nx
        self.ps = self.nb * per
        self.f_in = torch.empty(9 * self.ps, device=device)
        self.f_tg = torch.empty(9 * self.ps, device=device)
        rng = np.random.default_rng(seed)
        order = rng.permutation(nblk)
        tau_c = np.zeros(self.nb, np.float32)
        g_c = np.zeros(self.nb, np.float32)
        self.groups = []
        fine = L.shape(m * nx, m * h, per_group)
        ff = [torch.empty(9 * per_group * m * m * per, device=device) for _ in range(3)]
        nu_max = (2.0 - 0.5) / 3.0  # keeps tau_c < 2
        for gi in range(groups):
            u_ref = rng.uniform(*u_range)
            re_ref = float(np.exp(rng.uniform(np.log(re_range[0]), np.log(re_range[1]))))
            nu_ref = u_ref * h / re_ref
            g = 8.0 * nu_ref * u_ref / h ** 2
            s = np.exp(rng.uniform(-np.log(spread), np.log(spread), per_group))
            nu = np.minimum(nu_ref * s, nu_max)
            tc = (0.5 + 3.0 * nu).astype(np.float32)
            tf = (0.5 + m * (tc.astype(np.float64) - 0.5)).astype(np.float32)
            tf_d = torch.from_numpy(tf).to(device)
            tc_d = torch.from_numpy(tc).to(device)
            efold = h * h / (np.pi ** 2 * nu_ref)
            times = sorted({max(1, int(round(fr * efold))) for fr in snaps})
            while len(times) < len(snaps):       # short e-folding times: distinct steps
                times.append(times[-1] + 1)
            self.groups.append({"u_ref": u_ref, "re_ref": re_ref, "force": g,
                                "tau_c": tc.tolist(), "times": times})
            L.lbm_init_tgv(ff[0], fine, 1.0, 0.0, 0.0, 0.0, False)  # rest
            cur, done = 0, 0                     # fine steps taken
            for k, t in enumerate(times):
                blk = int(order[gi * len(snaps) + k])
                lo = blk * per_group
                tau_c[lo:lo + per_group] = tc
                g_c[lo:lo + per_group] = g
                coarse = L.shape(nx, h, per_group, self.ps)
                view = slice(lo * per, None)
                target = m * t - 1                   # fine state before coarse step t
                cur, done = self._run(ff, cur, fine, tf_d, g / m, target - done), target
                L.lbm_restrict_channel(ff[cur], fine, self.f_in[view], coarse, m, 0.0, tf_d, 0.0,
                                       tc_d, g / m)
                cur, done = self._run(ff, cur, fine, tf_d, g / m, m), done + m
                L.lbm_restrict_channel(ff[cur], fine, self.f_tg[view], coarse, m, 0.0, tf_d, 0.0,
                                       tc_d, g / m)
        self.tau_c = torch.from_numpy(tau_c).to(device)
        self.force = torch.from_numpy(g_c).to(device)

    @staticmethod
    def _run(ff, cur, fine, taus, g, steps):
        """`steps` fine channel steps from ff[cur]; returns the index of the
        buffer holding the result (ff[2] is the scratch of multi-step runs)."""
        if steps <= 0:
            return cur
        out = 1 - cur
        L.lbm_step_channel(ff[cur], ff[out], ff[2], fine, 0.0, taus, g, steps)
        return out

    def batch_view(self, j, batch):
        """(f_in, f_target, shape, taus, forces) of lattices batch*j ..
        batch*(j+1)-1: views into the bank with its plane stride."""
        lo = j * batch
        per = self.h * self.nx
        s = L.shape(self.nx, self.h, batch, self.ps)
        return (self.f_in[lo * per:], self.f_tg[lo * per:], s, self.tau_c[lo:lo + batch],
                self.force[lo:lo + batch])


class ChannelTrainer:
    """AdamW training of the channel network on a ChannelPairBank (fused C
    ABI step gnn_train_step_channel); epochs visit the bank's batches in a
    seeded random order.

    weighting: "eq4" (the paper's loss) or "relative" (each lattice weighted
    by mean(D) / D_b, capped at 1e4, with D_b its one-step residual under the
    BGK channel step: the zero network's loss on that lattice alone)."""

    def __init__(self, device, bank, theta=None, lr=1e-3, wd=1e-2, batch=64, seed=0,
                 weighting="eq4"):
        import torch
        if bank.nb % batch:
            raise ValueError("the bank must hold a whole number of batches")
        if weighting not in ("eq4", "relative"):
            raise ValueError(f"unknown weighting {weighting!r}")
        self.bank, self.batch = bank, batch
        theta = inputs.xavier_params(seed) if theta is None else theta
        self.params = torch.from_numpy(np.asarray(theta, np.float32)).to(device)
        self.packed = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=device)
        L.gnn_pack(self.params, self.packed)
        self.m = torch.zeros(L.gnn_trainable_count(), device=device)
        self.v = torch.zeros_like(self.m)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.ws = torch.empty(L.gnn_train_workspace_bytes(bank.batch_view(0, batch)[2]),
                              dtype=torch.uint8, device=device)
        self.lr, self.wd = lr, wd
        self.rng = np.random.default_rng(seed)
        self.queue = []
        self.step_count = 0
        self.lat_w = None
        if weighting == "relative":
            d = self.lattice_residuals(bank)
            w = np.where(d * 1e4 > d.mean(), d.mean() / np.where(d > 0, d, 1.0), 1e4)
            self.lat_w = torch.from_numpy(w.astype(np.float32)).to(device)

    def lattice_residuals(self, bank):
        """D_b of every lattice of `bank`: the zero network's Eq. 4 loss on
        that lattice alone (the BGK channel step's one-step residual)."""
        import torch
        zero = torch.from_numpy(inputs.zero_params()).to(self.m.device)
        pk = torch.empty_like(self.packed)
        L.gnn_pack(zero, pk)
        m, v = torch.zeros_like(self.m), torch.zeros_like(self.v)
        loss = torch.zeros(1, dtype=torch.float64, device=self.m.device)
        ws = torch.empty(L.gnn_train_workspace_bytes(bank.batch_view(0, 1)[2]), dtype=torch.uint8,
                         device=self.m.device)
        out = torch.empty(bank.nb, dtype=torch.float64, device=self.m.device)
        for j in range(bank.nb):
            f_in, f_tg, s, taus, forces = bank.batch_view(j, 1)
            L.gnn_train_step_channel(f_in, f_tg, s, 0.0, taus, 0.0, forces, None, zero, pk, m, v,
                                     1, 0.0, 0.0, loss, None, ws)
            out[j:j + 1].copy_(loss)
        return out.cpu().numpy()

    def step(self):
        if not self.queue:
            self.queue = list(self.rng.permutation(self.bank.nb // self.batch))
        j = int(self.queue.pop())
        f_in, f_tg, s, taus, forces = self.bank.batch_view(j, self.batch)
        lw = None if self.lat_w is None else self.lat_w[j * self.batch:(j + 1) * self.batch]
        self.step_count += 1
        L.gnn_train_step_channel(f_in, f_tg, s, 0.0, taus, 0.0, forces, lw, self.params,
                                 self.packed, self.m, self.v, self.step_count, self.lr, self.wd,
                                 self.loss, None, self.ws)

    def bank_loss(self, bank, params=None):
        """Mean Eq. 4 loss of `params` (device FP32; default: the trained
        ones) over every batch of `bank`, through the same fused step with
        lr = 0 and scratch moments, so that no parameter changes."""
        import torch
        params = self.params if params is None else params
        pk = torch.empty_like(self.packed)
        L.gnn_pack(params, pk)
        m, v = torch.zeros_like(self.m), torch.zeros_like(self.v)
        loss = torch.zeros(1, dtype=torch.float64, device=self.m.device)
        nbat = bank.nb // self.batch
        tot = 0.0
        for j in range(nbat):
            f_in, f_tg, s, taus, forces = bank.batch_view(j, self.batch)
            L.gnn_train_step_channel(f_in, f_tg, s, 0.0, taus, 0.0, forces, None, params, pk, m, v,
                                     1, 0.0, 0.0, loss, None, self.ws)
            tot += loss.item()
        return tot / nbat

    def theta(self):
        return self.params.cpu().numpy().copy()
