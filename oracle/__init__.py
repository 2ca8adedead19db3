"""Plain FP64 CPU oracle for LBM-GNN (arXiv 2504.14494).

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
restatement of the method that the CUDA path is checked against.  Only the
test suite, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline and
reference arms) may import it.  The product path (``paper_2504_14494_gb300``)
never imports it and shares no code, constant table or helper with it.

Modules:
  lbm    -- D2Q9 lattice, equilibrium (Eq. 2), BGK collision (Eq. 1),
            streaming, Taylor-Green vortex initial state and closed-form decay,
            domain totals (Sec. 2.1, Fig. 1, Sec. 3.2, Eq. 6).
  gnn    -- the GNN-enhanced collision (Sec. 2.2-2.3, Eq. 3, Fig. 2): feature
            extraction, encoder, message passing over the 8 lattice neighbours,
            tau-adjustment and delta-f heads, and its hand-derived backward.
  train  -- training-data restriction from a refined lattice, the MSE loss
            (Eq. 4) and the AdamW update (Sec. 2.4).

Everything is numpy float64 unless a docstring says otherwise.  Where the
paper is silent the reading taken is stated in the docstring of the function
that depends on it.
"""
