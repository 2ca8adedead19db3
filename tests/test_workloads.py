"""The workload records the benchmark reads: sizes, relaxation times and the
Reynolds numbers they imply (Re = u0 N / nu, nu = (tau - 1/2) / 3)."""
import pytest

from paper_2504_14494_gb300 import inputs, workloads as W


def test_tgv_records():
    assert (W.TGV_64.n, W.TGV_64.tau, W.TGV_64.u0, W.TGV_64.steps) == (64, 0.8, 0.01, 1000)
    assert W.TGV_4096.n == 4096 and W.TGV_4096.steps == 10000
    assert W.TGV_4096.re() == pytest.approx(2048.0)
    assert [round(W.TGV_4096.re(t)) for t in W.TGV_4096.tau_sweep] == [2048, 10007, 1228800]


def test_gnn_and_training_records():
    assert W.TGV_GNN_1024.tau == pytest.approx(0.6536)   # Re 1000 at u0 0.05 on 1024^2
    T = W.TRAIN_64x256
    assert (T.n, T.batch, T.refine, T.lr, T.weight_decay) == (256, 64, 4, 1e-3, 1e-2)


def test_batch_record_draws_the_serving_mix():
    B = W.BATCH_512
    d = inputs.batch_lattices(B.lattices, B.seed, B.side_lo, B.side_hi, B.re_lo, B.re_hi)
    assert len(d) == 512 and sum(x["gnn"] for x in d) == 256
    assert all(B.side_lo <= x["side"] <= B.side_hi for x in d)
    assert all(B.re_lo <= x["re"] <= B.re_hi for x in d)
    assert d == inputs.batch_lattices(512, 7)   # the defaults are the same draw


def test_training_instance_ranges():
    """The training draws: defaults u0 ~ U[0.01, 0.08], Re ~ U[100, 5000]
    (unchanged by the range arguments), and the high-Re recipe of the
    stability sweep (u0 ~ U[0.1, 0.3], Re log-uniform in [400, 51200])."""
    import numpy as np
    d = inputs.training_instances(2000, 3, 64)
    assert d == inputs.training_instances(2000, 3, 64, (0.01, 0.08), (100.0, 5000.0))
    assert all(0.01 <= x["u0"] <= 0.08 and 100.0 <= x["re"] <= 5000.0 for x in d)
    assert all(x["nu"] == pytest.approx(x["u0"] * 64 / x["re"]) for x in d)
    assert {x["k_mult"] for x in d} == {1, 2, 4}
    h = inputs.training_instances(2000, 3, 64, (0.1, 0.3), (400.0, 51200.0), log_re=True)
    re = np.array([x["re"] for x in h])
    assert re.min() >= 400.0 and re.max() <= 51200.0
    # log-uniform: each factor-2 band of the 7 between 400 and 51200 holds ~1/7
    counts = np.histogram(np.log2(re / 400.0), bins=7, range=(0, 7))[0]
    assert counts.min() > 200 and counts.max() < 380
    assert all(0.1 <= x["u0"] <= 0.3 for x in h)
