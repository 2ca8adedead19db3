"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.

This module holds no arithmetic of the method: it draws random numbers and
lays them out (weights, perturbations, per-instance flow parameters, lattice
sizes).  Everything the method computes lives in the CUDA library (and,
independently, in the test oracle).

Parameter vector layout (float32), shared as an interface by the CUDA library
and the oracle:
  enc1.W[64,12] enc1.b[64] enc2.W[64,64] enc2.b[64]
  {edge.W[64,130] edge.b[64] node.W[64,128] node.b[64]} x 2 rounds
  head.W[10,64] head.b[10]                      -> 38,922 trainable values
  mu[12] sigma[12] s_df variant                 -> 26 fixed values
variant: 0, or a sum of flags: 1 = MLP-only network of the paper's Fig. 2
(ReLU encoder, no message passing), 2 = mass/momentum-conserving correction,
4 = relaxation-time head unused (tau_adj = 1).
"""
import numpy as np

HID, NFEAT, NOUT, ROUNDS = 64, 12, 10, 2
PARAM_SHAPES = [(HID, NFEAT), (HID,), (HID, HID), (HID,)]
for _ in range(ROUNDS):
    PARAM_SHAPES += [(HID, 2 * HID + 2), (HID,), (HID, 2 * HID), (HID,)]
PARAM_SHAPES += [(NOUT, HID), (NOUT,)]
N_TRAINABLE = sum(int(np.prod(s)) for s in PARAM_SHAPES)
N_PARAMS = N_TRAINABLE + 2 * NFEAT + 2
MLP_ONLY, CONSERVATIVE, FIXED_TAU = 1, 2, 4

# Default input normaliser: populations around their rest-state values
# (4/9, 1/9 x4, 1/36 x4) with a 10% scale, density around 1, velocity with a
# 0.01 scale; default output scale of the Delta-f head.
_REST = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
DEFAULT_MU = np.array(_REST + [1.0, 0.0, 0.0], dtype=np.float32)
DEFAULT_SIGMA = np.array([0.1 * w for w in _REST] + [0.01, 0.01, 0.01], dtype=np.float32)
DEFAULT_S_DF = 1e-4


def xavier_params(seed, s_df=DEFAULT_S_DF, mu=None, sigma=None, weight_gain=1.0,
                  bias_scale=0.0, variant=0):
    """Xavier-uniform weights (bound gain*sqrt(6/(fan_in+fan_out))), biases
    zero (or uniform in +-bias_scale), from numpy's PCG64 seeded by `seed`."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in PARAM_SHAPES:
        if len(s) == 2:
            bound = weight_gain * np.sqrt(6.0 / (s[0] + s[1]))
            parts.append(rng.uniform(-bound, bound, size=s).astype(np.float32).ravel())
        else:
            parts.append(rng.uniform(-bias_scale, bias_scale, size=s).astype(np.float32)
                         if bias_scale > 0 else np.zeros(s, np.float32))
    parts.append(DEFAULT_MU if mu is None else np.asarray(mu, np.float32))
    parts.append(DEFAULT_SIGMA if sigma is None else np.asarray(sigma, np.float32))
    parts.append(np.array([s_df, float(variant)], np.float32))
    out = np.concatenate(parts).astype(np.float32)
    assert out.shape == (N_PARAMS,)
    return out


def zero_params(s_df=DEFAULT_S_DF, variant=0):
    """All trainable values zero; default normaliser."""
    out = np.zeros(N_PARAMS, np.float32)
    out[N_TRAINABLE:N_TRAINABLE + NFEAT] = DEFAULT_MU
    out[N_TRAINABLE + NFEAT:N_TRAINABLE + 2 * NFEAT] = DEFAULT_SIGMA
    out[-2] = s_df
    out[-1] = float(variant)
    return out


def perturbation(shape, seed, amplitude):
    """Multiplicative noise 1 + amplitude*U(-1, 1) of the given shape."""
    rng = np.random.default_rng(seed)
    return (1.0 + amplitude * rng.uniform(-1.0, 1.0, size=shape)).astype(np.float64)


def normal(shape, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    return (scale * rng.standard_normal(shape)).astype(np.float64)


def training_instances(n, seed, n_coarse=256, u0_range=(0.01, 0.08), re_range=(100.0, 5000.0),
                       log_re=False):
    """Per-instance TGV draws of the training workload: k multiple in
    {1, 2, 4}, u0 ~ U[u0_range] (default [0.01, 0.08]), Re ~ U[re_range]
    (default [100, 5000]; log-uniform with log_re).  Returns a list of dicts
    with the lattice viscosity from Re = u0 N / nu (tau follows from nu)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        kmult = int(rng.choice([1, 2, 4]))
        u0 = float(rng.uniform(*u0_range))
        if log_re:
            re = float(np.exp(rng.uniform(np.log(re_range[0]), np.log(re_range[1]))))
        else:
            re = float(rng.uniform(*re_range))
        nu = u0 * n_coarse / re
        out.append({"k_mult": kmult, "u0": u0, "re": re, "nu": nu})
    return out


def batch_lattices(n, seed, side_lo=32, side_hi=1024, re_lo=100.0, re_hi=5000.0):
    """Lattice draws of the batched serving workload: square sides
    log-uniform in [side_lo, side_hi] (rounded), Re ~ U[re_lo, re_hi],
    u0 ~ U[0.01, 0.08], first half plain BGK and second half GNN."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        side = int(round(float(np.exp(rng.uniform(np.log(side_lo), np.log(side_hi))))))
        u0 = float(rng.uniform(0.01, 0.08))
        re = float(rng.uniform(re_lo, re_hi))
        out.append({"side": side, "u0": u0, "re": re, "nu": u0 * side / re,
                    "gnn": i >= n // 2})
    return out
