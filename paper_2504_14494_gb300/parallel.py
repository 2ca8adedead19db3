"""Multi-rank execution: one process per GPU, torch.distributed for the
little that crosses ranks.

The method's work splits into independent units, so no step of a lattice
update exchanges data between ranks:

  * stepping (plain BGK, GNN-LBM, batched lattices): each rank advances its
    own lattices.  The only cross-rank operation is the host-side
    aggregation of a timed region: the slowest rank's time and the units
    summed over ranks (`aggregate_throughput`).  Lattices of uneven size are
    dealt to ranks by `shard` (longest-processing-time first).
  * training (Sec. 2.4): data parallel over training instances.  Every rank
    computes the gradient of Eq. 4 on its own pairs; one all-reduce of the
    38,922 FP32 gradient values per step averages them (with equal node
    counts per rank the average is the gradient of the mean over the union of
    the ranks' pairs), then every rank applies the same AdamW update, so the
    parameter vectors stay identical.

  * one large lattice split over ranks (`SlabLattice`): each rank owns a slab
    of rows plus `halo` ghost rows on each side; a step is one ghost-row
    exchange with the two neighbouring ranks (the only data-path
    communication: 9 x halo x nx values each way) followed by the ordinary
    periodic step on the padded slab, which leaves every owned row exact
    (the step reads rows at most `halo` away: 1 for BGK, 3 for the GNN step,
    which streams and then passes messages twice) and only the ghost rows
    stale until the next exchange.  The domain totals are one FP64
    all-reduce of the ranks' owned-row totals.

Every function here works with world size 1 (no process group) and with any
backend; the host logic is exercised with `gloo` on CPU tensors.
"""
import numpy as np

from . import inputs
from . import lib as L


def _dist():
    import torch.distributed as dist
    return dist if dist.is_available() and dist.is_initialized() else None


def rank_and_size(group=None):
    """(rank, world size) in `group`; (0, 1) without a process group."""
    dist = _dist()
    if dist is None:
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def shard(weights, size):
    """Deal units of the given weights (e.g. node counts) to `size` ranks:
    heaviest first, each to the currently lightest rank (lowest rank on
    ties).  Deterministic; returns one sorted index list per rank.  The
    heaviest rank carries at most the mean load plus the largest unit."""
    if size < 1:
        raise ValueError("size must be >= 1")
    w = [float(x) for x in weights]
    if any(x < 0 for x in w):
        raise ValueError("weights must be non-negative")
    order = sorted(range(len(w)), key=lambda i: (-w[i], i))
    load = [0.0] * size
    out = [[] for _ in range(size)]
    for i in order:
        r = min(range(size), key=lambda j: (load[j], j))
        out[r].append(i)
        load[r] += w[i]
    return [sorted(o) for o in out]


def average_(t, group=None):
    """In-place mean of tensor `t` over the ranks of `group` (no-op alone)."""
    dist = _dist()
    if dist is None:
        return t
    size = dist.get_world_size(group)
    if size > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        t.div_(size)
    return t


def broadcast_(t, src=0, group=None):
    """In-place copy of rank `src`'s tensor to every rank of `group`."""
    dist = _dist()
    if dist is not None and dist.get_world_size(group) > 1:
        dist.broadcast(t, src=src, group=group)
    return t


def aggregate_throughput(units, ms, device="cpu", group=None):
    """Host aggregation of a timed region.  `units`: work this rank did
    (e.g. node updates); `ms`: its measured time.  Returns
    (units summed over ranks, slowest rank's ms, summed units per second)."""
    import torch
    dist = _dist()
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if dist is not None and dist.get_world_size(group) > 1:
        dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    total, t_max = float(u.item()), float(t.item())
    return total, t_max, (total / (t_max / 1e3) if t_max > 0 else float("inf"))


class DataParallelTrainer:
    """AdamW training of the network, data parallel over ranks.

    Per step and rank: the next batch of pairs from this rank's PairStream
    (instances seeded by `seed` and the rank), then through the C ABI
    lbm_stream, gnn_forward, gnn_collide_loss (Eq. 3, Eq. 4, dL/dy) and
    gnn_backward (dL/dparams); the gradient and the loss are averaged over
    ranks (`average_`), and gnn_adamw plus gnn_pack update every rank's
    identical parameter copy.  With one rank this is the same computation as
    the fused gnn_train_step."""

    def __init__(self, device, theta=None, lr=1e-3, wd=1e-2, seed=0, group=None, **stream_kw):
        import torch
        from .train import PairStream
        self.group = group
        self.rank, self.size = rank_and_size(group)
        self.data = PairStream(device, seed=seed * 1009 + self.rank, **stream_kw)
        theta = inputs.xavier_params(seed) if theta is None else theta
        self.params = torch.from_numpy(np.asarray(theta, np.float32)).to(device)
        broadcast_(self.params, 0, group)
        s = self.data.coarse
        n = s.nx * s.ny * s.nb
        nt = L.gnn_trainable_count()
        self.packed = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=device)
        L.gnn_pack(self.params, self.packed)
        self.m = torch.zeros(nt, device=device)
        self.v = torch.zeros_like(self.m)
        self.grads = torch.zeros(nt, device=device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=device)
        self.f_pre = torch.empty(9 * n, device=device)
        self.y = torch.empty(10 * n, device=device)
        self.dy = torch.empty(10 * n, device=device)
        self.saved = torch.empty(L.gnn_saved_bytes(s), dtype=torch.uint8, device=device)
        self.ws_loss = torch.empty(L.gnn_loss_workspace_bytes(s), dtype=torch.uint8,
                                   device=device)
        self.ws_bwd = torch.empty(L.gnn_backward_workspace_bytes(s), dtype=torch.uint8,
                                  device=device)
        self.lr, self.wd = lr, wd
        self.step_count = 0

    def step(self):
        """One data-parallel step; returns nothing (the rank-averaged loss
        before the update is left in self.loss)."""
        s = self.data.coarse
        f_in, f_tg, tau_c = self.data.next()
        self.step_count += 1
        L.lbm_stream(f_in, self.f_pre, s)
        L.gnn_forward(self.f_pre, s, self.packed, self.saved, self.y)
        L.gnn_collide_loss(self.f_pre, self.y, f_tg, s, 1.0, tau_c, self.packed, self.loss,
                           self.dy, None, self.ws_loss)
        L.gnn_backward(self.f_pre, s, self.packed, self.saved, self.dy, self.grads, None,
                       self.ws_bwd)
        average_(self.grads, self.group)
        average_(self.loss, self.group)
        L.gnn_adamw(self.params, self.grads, self.m, self.v, self.step_count, self.lr, self.wd)
        L.gnn_pack(self.params, self.packed)

    def theta(self):
        return self.params.cpu().numpy().copy()


def _device_totals(view):
    """lbm_moments totals of a [9, rows, nx] FP32 device view whose planes
    are strided (rows contiguous within a plane)."""
    import torch
    q, rows, nx = view.shape
    assert view.stride(2) == 1 and view.stride(1) == nx, "rows must be contiguous"
    out = torch.zeros(5, dtype=torch.float64, device=view.device)
    L.lbm_moments(view.data_ptr(), L.shape(nx, rows, 1, view.stride(0)), None, None, None, out)
    return out


# D2Q9 populations that cross a row boundary of the slab in one streaming
# step: e_y = +1 (moving up: read by the row above from the row below) and
# e_y = -1 (moving down).
CROSS_UP = (2, 5, 6)
CROSS_DOWN = (4, 7, 8)
NOT_UP = tuple(q for q in range(9) if q not in CROSS_UP)
NOT_DOWN = tuple(q for q in range(9) if q not in CROSS_DOWN)


class SlabLattice:
    """One periodic nx x ny lattice split into row slabs over the ranks of
    `group`: rank r owns rows [ny r / P, ny (r + 1) / P) and keeps them with
    `halo` ghost rows below and above in a [9, rows + 2 halo, nx] tensor
    (`f`).  `step(step_fn)` exchanges the ghost rows with the neighbouring
    ranks (periodic in y) and applies step_fn, a periodic step on a
    [9, R, nx] population tensor returning the stepped tensor.  With one
    rank the ghost rows come from the slab's own periodic wrap.

    With one ghost row (the BGK step: streaming is the only coupling between
    rows) only the 3 populations that stream across each face are exchanged
    (`faces_only`, the default for halo 1): the owned rows read nothing else
    from the ghost rows.  The other 6 populations of each ghost row are
    filled locally from the adjacent owned row, so the ghost rows that
    step_fn also steps hold plausible, finite states.  With more ghost rows
    (the GNN step reads all populations of nodes up to 3 rows away) all 9
    populations are exchanged."""

    def __init__(self, nx, ny, halo, device="cpu", dtype=None, group=None, faces_only=None):
        import torch
        self.group = group
        self.rank, self.size = rank_and_size(group)
        self.nx, self.ny, self.halo = nx, ny, halo
        self.faces_only = (halo == 1) if faces_only is None else bool(faces_only)
        if self.faces_only and halo != 1:
            raise ValueError("faces_only needs exactly one ghost row")
        self.r0 = ny * self.rank // self.size
        self.r1 = ny * (self.rank + 1) // self.size
        self.rows = self.r1 - self.r0
        if self.rows < halo:
            raise ValueError("every rank needs at least `halo` rows")
        self.f = torch.zeros((9, self.rows + 2 * halo, nx), device=device,
                             dtype=dtype or torch.float32)

    def load(self, full):
        """Owned rows from a full [9, ny, nx] state (a tensor on any device)."""
        self.f[:, self.halo:self.halo + self.rows] = full[:, self.r0:self.r1].to(self.f)

    def interior(self):
        return self.f[:, self.halo:self.halo + self.rows]

    def exchange(self):
        """Ghost rows below <- the previous rank's top `halo` owned rows,
        ghost rows above <- the next rank's bottom `halo` owned rows (with
        `faces_only`: the 3 populations crossing each face, 3 x nx values
        each way instead of 9 x nx)."""
        import torch
        h, R = self.halo, self.rows
        if self.faces_only:
            up, down = list(CROSS_UP), list(CROSS_DOWN)
            top = self.f[up, R:R + 1].contiguous()       # moving up out of my top row
            bottom = self.f[down, 1:2].contiguous()      # moving down out of my bottom row
            # the rest of each ghost row: a local copy of the adjacent owned row
            self.f[list(NOT_UP), 0:1] = self.f[list(NOT_UP), 1:2]
            self.f[list(NOT_DOWN), R + 1:R + 2] = self.f[list(NOT_DOWN), R:R + 1]
        else:
            top = self.f[:, R:R + h].contiguous()        # my top owned rows
            bottom = self.f[:, h:2 * h].contiguous()      # my bottom owned rows
        gsel = (list(CROSS_UP), list(CROSS_DOWN)) if self.faces_only else (slice(None),) * 2
        dist = _dist()
        if dist is None or self.size == 1:
            self.f[gsel[0], :h] = top
            self.f[gsel[1], R + h:] = bottom
            return
        prev = (self.rank - 1) % self.size
        nxt = (self.rank + 1) % self.size
        below = torch.empty_like(top)
        above = torch.empty_like(bottom)
        ops = [dist.P2POp(dist.isend, top, nxt, self.group, 0),
               dist.P2POp(dist.isend, bottom, prev, self.group, 1),
               dist.P2POp(dist.irecv, below, prev, self.group, 0),
               dist.P2POp(dist.irecv, above, nxt, self.group, 1)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        self.f[gsel[0], :h] = below
        self.f[gsel[1], R + h:] = above

    def step(self, step_fn):
        self.exchange()
        self.f = step_fn(self.f)

    def totals(self, moments_fn=None):
        """FP64 domain totals of the whole lattice (mass, x- and y-momentum,
        kinetic energy, non-finite node count; the quantities of
        lbm_moments): each rank's totals over its owned rows, summed over
        ranks by one FP64 all-reduce.  moments_fn(view) -> float64 tensor[5]
        computes them for a [9, rows, nx] view of the owned rows (a strided
        view into the padded slab); default: lbm_moments through the C ABI
        on that view in place (plane stride of the padded slab)."""
        import torch
        view = self.interior()
        if moments_fn is None:
            moments_fn = _device_totals
        t = moments_fn(view).to(torch.float64)
        dist = _dist()
        if dist is not None and self.size > 1:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t

    def gather(self):
        """The full [9, ny, nx] state on every rank (all-gather of the slabs)."""
        import torch
        dist = _dist()
        mine = self.interior().contiguous()
        if dist is None or self.size == 1:
            return mine.clone()
        counts = [self.ny * (r + 1) // self.size - self.ny * r // self.size
                  for r in range(self.size)]
        width = max(counts)  # all-gather wants equal shapes: pad the slabs
        padded = torch.zeros((9, width, self.nx), device=mine.device, dtype=mine.dtype)
        padded[:, :self.rows] = mine
        parts = [torch.empty_like(padded) for _ in counts]
        dist.all_gather(parts, padded, group=self.group)
        return torch.cat([p[:, :c] for p, c in zip(parts, counts)], dim=1)

