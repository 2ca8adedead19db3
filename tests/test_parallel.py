"""Multi-rank host logic (paper_2504_14494_gb300.parallel) on CPU: sharding
of uneven lattices, and two `gloo` ranks for the gradient average, the
parameter broadcast and the timing aggregation of the benchmark.  The
data-parallel gradient is checked against the FP64 oracle's gradient of the
Eq. 4 loss over the union of both ranks' lattices."""
import datetime
import os
import socket

import numpy as np
import pytest

from paper_2504_14494_gb300 import inputs, parallel


def test_shard_is_a_balanced_partition():
    rng = np.random.default_rng(5)
    for size in (1, 2, 3, 5, 8):
        for n in (0, 1, 7, 64):
            w = rng.integers(0, 1000, size=n).astype(float)
            parts = parallel.shard(w, size)
            assert len(parts) == size
            flat = sorted(i for p in parts for i in p)
            assert flat == list(range(n))
            if n:
                loads = [sum(w[i] for i in p) for p in parts]
                assert max(loads) <= w.sum() / size + w.max() + 1e-9
            assert parts == parallel.shard(list(w), size)  # deterministic


def test_shard_of_the_batched_workload():
    """The 512 uneven lattices of the batched serving workload over 4 ranks:
    every rank within 1% of the mean node count."""
    lat = inputs.batch_lattices(512, 7)
    w = [d["side"] ** 2 for d in lat]
    parts = parallel.shard(w, 4)
    loads = np.array([sum(w[i] for i in p) for p in parts], float)
    assert loads.max() / loads.mean() < 1.01


def test_shard_rejects_bad_arguments():
    with pytest.raises(ValueError):
        parallel.shard([1, 2], 0)
    with pytest.raises(ValueError):
        parallel.shard([1, -2], 2)


def test_without_process_group_everything_is_local():
    torch = pytest.importorskip("torch")
    t = torch.tensor([1.0, 2.0])
    assert parallel.rank_and_size() == (0, 1)
    assert parallel.average_(t) is t and t.tolist() == [1.0, 2.0]
    assert parallel.broadcast_(t) is t and t.tolist() == [1.0, 2.0]
    total, t_max, rate = parallel.aggregate_throughput(50, 10.0)
    assert (total, t_max) == (50.0, 10.0) and rate == pytest.approx(5000.0)


def _lattice(rank):
    from oracle import lbm
    nx, ny = 6, 5
    f = lbm.tgv_init(nx, ny, 1.0, 0.04, 2 * np.pi / nx, 2 * np.pi / ny)
    return f * inputs.perturbation(f.shape, 100 + rank, 2e-2)


def _oracle_grad(f_post, theta, tau):
    """FP64 oracle gradient (trainable order) of the Eq. 4 loss of one
    GNN-LBM step of f_post against a target drawn from the seed."""
    from oracle import gnn, lbm
    p = gnn.unpack(theta)
    f_pre = lbm.stream_pull(f_post)
    y, cache = gnn.forward(f_pre, p)
    target = lbm.bgk_step(f_post, tau) * inputs.perturbation(f_post.shape, 7, 1e-3)
    loss, dy, _ = gnn.collide_loss(f_pre, y, tau, target, p)
    g, _ = gnn.backward(dy, cache, p)
    return loss, gnn.pack_grads(g)


def _worker(rank, port, size):
    import torch
    import torch.distributed as dist
    from oracle import train as otrain
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=size, timeout=datetime.timedelta(seconds=60))
    try:
        assert parallel.rank_and_size() == (rank, size)
        t = torch.tensor([rank + 1.0, 10.0 * (rank + 1)], dtype=torch.float64)
        parallel.average_(t)
        assert t.tolist() == [1.5, 15.0]
        b = torch.full((3,), float(rank))
        parallel.broadcast_(b, src=0)
        assert b.tolist() == [0.0, 0.0, 0.0]
        total, t_max, rate = parallel.aggregate_throughput(100 * (rank + 1), 10.0 + rank)
        assert total == 300.0 and t_max == 11.0 and rate == pytest.approx(300.0 / 0.011)

        # Data-parallel gradient: each rank the Eq. 4 gradient of its own
        # lattice, averaged; equal node counts, so the average is the
        # gradient of the mean over both lattices' nodes x 9.
        theta = inputs.xavier_params(3, s_df=1e-2, bias_scale=0.1)
        tau = 0.7
        loss, g = _oracle_grad(_lattice(rank), theta, tau)
        gt = torch.from_numpy(g.copy())
        lt = torch.tensor([loss], dtype=torch.float64)
        parallel.average_(gt)
        parallel.average_(lt)
        l0, g0 = _oracle_grad(_lattice(0), theta, tau)
        l1, g1 = _oracle_grad(_lattice(1), theta, tau)
        n0 = n1 = _lattice(0)[0].size
        want = (n0 * g0 + n1 * g1) / (n0 + n1)
        assert np.allclose(gt.numpy(), want, rtol=1e-12, atol=1e-18)
        assert lt.item() == pytest.approx((n0 * l0 + n1 * l1) / (n0 + n1), rel=1e-12)
        # the same update on every rank keeps the copies identical
        th = theta[:inputs.N_TRAINABLE].astype(np.float64)
        new, _, _ = otrain.adamw_step(th, gt.numpy(), np.zeros_like(th), np.zeros_like(th), 1,
                                      1e-3, 1e-2)
        mine = torch.from_numpy(new.copy())
        first = mine.clone()
        parallel.broadcast_(first, src=0)
        assert torch.equal(mine, first)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    ctx = mp.start_processes(_worker, args=(_free_port(), 2), nprocs=2, join=False,
                             start_method="spawn")
    import time
    deadline = time.monotonic() + 300
    while not ctx.join(timeout=5):  # False while a rank is still running
        if time.monotonic() > deadline:
            for p in ctx.processes:
                p.kill()
            pytest.fail("the gloo ranks did not finish within 300 s")


def _oracle_step_fn(kind, theta=None, tau=0.7):
    """A periodic step on a [9, R, nx] torch tensor through the oracle."""
    import torch
    from oracle import gnn, lbm

    def fn(f):
        a = f.numpy()
        out = lbm.bgk_step(a, tau) if kind == "bgk" else gnn.gnn_step(a, theta, tau)
        return torch.from_numpy(np.ascontiguousarray(out))
    return fn


def _full_state(nx, ny, seed):
    from oracle import lbm
    f = lbm.tgv_init(nx, ny, 1.0, 0.04, 2 * np.pi / nx, 2 * np.pi / ny)
    return f * inputs.perturbation(f.shape, seed, 2e-2)


def _slab_worker(rank, port, size, result_q):
    import torch
    import torch.distributed as dist
    from oracle import gnn, lbm
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=size, timeout=datetime.timedelta(seconds=60))
    try:
        full = _full_state(12, 10, 3)
        theta = inputs.xavier_params(5, s_df=1e-2, bias_scale=0.1)
        for kind, halo, steps in (("bgk", 1, 4), ("gnn", 3, 2)):
            slab = parallel.SlabLattice(12, 10, halo, dtype=torch.float64)
            slab.load(torch.from_numpy(full))
            for _ in range(steps):
                slab.step(_oracle_step_fn(kind, theta))
            got = slab.gather().numpy()
            ref = full
            for _ in range(steps):
                ref = lbm.bgk_step(ref, 0.7) if kind == "bgk" else gnn.gnn_step(ref, theta, 0.7)
            if kind == "bgk":
                assert np.array_equal(got, ref), kind   # the same FP64 operations per node
            else:
                assert np.allclose(got, ref, rtol=1e-12, atol=1e-15), kind
            # domain totals: owned-row totals of every rank, one FP64 all-reduce
            tot = slab.totals(lambda v: torch.tensor(np.asarray(lbm.totals(v.numpy()), float)))
            want = np.asarray(lbm.totals(ref), float)
            assert np.allclose(tot.numpy()[:4], want[:4], rtol=1e-12, atol=1e-14), kind
            assert tot.numpy()[4] == want[4] == 0.0
        result_q.put((rank, "ok"))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("size", [1, 2, 3])
def test_slab_decomposition_equals_single_domain(size):
    """One 12 x 10 lattice split into row slabs over 1-3 gloo ranks: ghost-row
    exchange + the periodic step on each padded slab reproduces the
    single-domain oracle run (BGK: 1 ghost row, bitwise; GNN step: 3 ghost
    rows, to FP64 rounding of the batched matrix products), and the FP64
    all-reduce of the ranks' owned-row totals equals the totals of the whole
    lattice to summation-order rounding."""
    pytest.importorskip("torch")
    import time
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    procs = mp.start_processes(_slab_worker, args=(_free_port(), size, q), nprocs=size,
                               join=False, start_method="spawn")
    deadline = time.monotonic() + 300
    while not procs.join(timeout=5):
        if time.monotonic() > deadline:
            for p in procs.processes:
                p.kill()
            pytest.fail("the gloo ranks did not finish within 300 s")
    got = sorted(q.get() for _ in range(size))
    assert got == [(r, "ok") for r in range(size)]

