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
