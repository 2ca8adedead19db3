"""The benchmark workloads as plain configuration records, with their seeds
written out; bench.py reads its sizes, relaxation times and seeds from here.

Every input is synthetic: Taylor-Green vortices (Sec. 3.2) initialised by the
library, random draws from numpy PCG64 seeded as stated.  Re = u0 N / nu
with nu = (tau - 1/2) / 3 in lattice units.
"""
from dataclasses import dataclass


@dataclass(frozen=True)
class TgvBgk:
    """Plain BGK Taylor-Green vortex on an n x n periodic lattice."""
    n: int
    tau: float
    u0: float
    steps: int
    tau_sweep: tuple = ()

    @property
    def k(self):
        import math
        return 2 * math.pi / self.n

    def re(self, tau=None):
        return self.u0 * self.n / (((self.tau if tau is None else tau) - 0.5) / 3.0)


@dataclass(frozen=True)
class TgvGnn:
    """GNN-corrected collision inference on an n x n TGV at Reynolds number
    `re` (tau from Re = u0 n / nu); untrained weights Xavier-uniform with
    `weight_seed`."""
    n: int
    re: float
    u0: float
    weight_seed: int

    @property
    def tau(self):
        return 0.5 + 3.0 * self.u0 * self.n / self.re


@dataclass(frozen=True)
class Training:
    """Training on library-generated pairs: `batch` TGV instances of n x n
    coarse nodes (k multiple in {1, 2, 4}, u0 ~ U[0.01, 0.08], Re ~
    U[100, 5000]), refined `refine` times; AdamW."""
    n: int
    batch: int
    refine: int
    lr: float
    weight_decay: float
    seed: int
    episode: int


@dataclass(frozen=True)
class BatchServing:
    """`lattices` TGVs, sides log-uniform in [side_lo, side_hi], Re ~
    U[re_lo, re_hi], u0 ~ U[0.01, 0.08]; first half BGK, second half GNN;
    `steps` steps as one graph launch."""
    lattices: int
    seed: int
    side_lo: int
    side_hi: int
    re_lo: float
    re_hi: float
    steps: int


# The five workloads the benchmark reports.
TGV_64 = TgvBgk(n=64, tau=0.8, u0=0.01, steps=1000)
TGV_4096 = TgvBgk(n=4096, tau=0.8, u0=0.05, steps=10000, tau_sweep=(0.8, 0.5614, 0.5005))
TGV_GNN_1024 = TgvGnn(n=1024, re=1000.0, u0=0.05, weight_seed=0)
TRAIN_64x256 = Training(n=256, batch=64, refine=4, lr=1e-3, weight_decay=1e-2, seed=1,
                        episode=64)
BATCH_512 = BatchServing(lattices=512, seed=7, side_lo=32, side_hi=1024, re_lo=100.0,
                         re_hi=5000.0, steps=1000)

ALL = {"tgv_bgk_64x64": TGV_64, "tgv_bgk_4096x4096": TGV_4096,
       "tgv_gnn_1024x1024": TGV_GNN_1024, "train_64x256x256_refined4": TRAIN_64x256,
       "batch_512_lattices_sides_32_1024": BATCH_512}
