"""gnn_params_init_xavier (host-side starting point of the parameter
vector, through the C ABI; no GPU needed): Xavier-uniform bounds and moments
per weight matrix, zero biases, the default input normaliser, determinism in
the seed, argument checks, and that the oracle runs the vector it makes."""
import numpy as np
import pytest

from paper_2504_14494_gb300 import inputs


def _init(L, seed, s_df=1e-4, variant=0):
    v = np.full(L.gnn_param_count(), np.nan, np.float32)
    return L.gnn_params_init_xavier(v, seed, s_df, variant)


def test_xavier_bounds_moments_and_fixed_values(lbmlib):
    L = lbmlib
    v = _init(L, 7, s_df=3e-4, variant=2)
    assert np.all(np.isfinite(v))
    off = 0
    for shape in inputs.PARAM_SHAPES:
        n = int(np.prod(shape))
        t = v[off:off + n].astype(np.float64)
        if len(shape) == 2:
            b = np.sqrt(6.0 / (shape[0] + shape[1]))
            assert np.all(np.abs(t) <= b), shape
            assert np.abs(t).max() > 0.95 * b, shape                 # the whole range is used
            assert abs(t.mean()) < 5 * b / np.sqrt(3 * n), shape     # U(-b, b): mean 0
            assert abs(t.var() / (b * b / 3) - 1) < 6 * np.sqrt(0.8 / n) + 0.02, shape
        else:
            assert np.all(t == 0), shape
        off += n
    assert off == inputs.N_TRAINABLE
    assert np.array_equal(v[off:off + 12], inputs.DEFAULT_MU)
    assert np.allclose(v[off + 12:off + 24], inputs.DEFAULT_SIGMA, rtol=1e-7)
    assert v[-2] == np.float32(3e-4) and v[-1] == 2.0


def test_seed_determinism(lbmlib):
    L = lbmlib
    a, b, c = _init(L, 11), _init(L, 11), _init(L, 12)
    assert np.array_equal(a, b)
    assert not np.array_equal(a[:inputs.N_TRAINABLE], c[:inputs.N_TRAINABLE])


def test_bad_arguments(lbmlib):
    L = lbmlib
    for s_df, variant in ((float("nan"), 0), (0.0, 0), (-1.0, 0), (1e-4, 8), (1e-4, -1)):
        with pytest.raises(L.LbmError, match="LBM_ERR_ARG"):
            _init(L, 1, s_df, variant)
    with pytest.raises(L.LbmError, match="LBM_ERR_ARG"):  # NULL vector
        L.check(L.load().gnn_params_init_xavier(None, 1, 1e-4, 0), "gnn_params_init_xavier")


def test_oracle_runs_the_vector(lbmlib):
    from oracle import gnn, lbm
    v = _init(lbmlib, 3, s_df=1e-3)
    f = lbm.tgv_init(6, 5, 1.0, 0.05, 2 * np.pi / 6, 2 * np.pi / 5)
    out = gnn.gnn_step(f, v, 0.7)
    assert out.shape == f.shape and np.all(np.isfinite(out))
