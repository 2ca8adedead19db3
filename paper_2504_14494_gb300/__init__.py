"""GB300-native (sm_103a) LBM-GNN: the D2Q9 BGK step and the GNN-enhanced
collision of arXiv 2504.14494 behind the C ABI of liblbmgnn.so.

  lib     -- ctypes binding, one Python function per C entry point
  build   -- in-tree nvcc build of liblbmgnn.so
  inputs  -- seeded synthetic inputs (weights, perturbations, workloads)
  autograd -- torch.autograd.Function over gnn_forward / gnn_backward
  train   -- refined-lattice training pairs and the fused training loop
  parallel -- multi-rank host logic: sharding, timing aggregation,
              data-parallel training (one gradient all-reduce per step)
  checkpoint -- CRC-checked save/restore of training state
  workloads -- the benchmark workloads (sizes, relaxation times, seeds)
"""
from . import lib  # noqa: F401
