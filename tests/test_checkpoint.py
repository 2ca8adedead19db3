"""Checkpoint format: round trip, CRC and header checks (CPU), and bitwise
resume of a GPU run (k steps, save, load, N - k steps == N steps)."""
import numpy as np
import pytest

from paper_2504_14494_gb300 import checkpoint


def test_round_trip_and_corruption(tmp_path):
    p = tmp_path / "a.ckpt"
    recs = {"f": np.arange(12, dtype=np.float32).reshape(3, 4), "step": np.int64(7),
            "tau": np.float64(0.8), "blob": np.arange(5, dtype=np.uint8)}
    checkpoint.save(p, recs)
    back = checkpoint.load(p)
    for k, v in recs.items():
        assert np.array_equal(back[k], v) and back[k].dtype == np.asarray(v).dtype
    raw = bytearray(p.read_bytes())
    raw[-1] ^= 0xFF
    p.write_bytes(bytes(raw))
    with pytest.raises(ValueError):
        checkpoint.load(p)
    p.write_bytes(b"XXXXXXXX" + bytes(raw[8:]))
    with pytest.raises(ValueError):
        checkpoint.load(p)


@pytest.mark.gpu
def test_resume_is_bitwise(lbmlib, cuda, tmp_path):
    import torch
    L = lbmlib
    n = 48
    s = L.shape(n, n)
    k = 2 * np.pi / n
    f0 = torch.empty(9 * n * n, device=cuda)
    L.lbm_init_tgv(f0, s, 1.0, 0.05, k, k, False)
    a, b, t = (torch.empty_like(f0) for _ in range(3))
    L.lbm_step_bgk(f0, a, t, s, 0.7, nsteps=30)                # uninterrupted
    L.lbm_step_bgk(f0, b, t, s, 0.7, nsteps=12)                # interrupted at 12
    p = tmp_path / "run.ckpt"
    checkpoint.save(p, {"f": b, "step": np.int64(12), "tau": np.float64(0.7)})
    c = torch.zeros_like(f0)
    rest = checkpoint.restore(p, {"f": c})
    assert int(rest["step"]) == 12
    d = torch.empty_like(f0)
    L.lbm_step_bgk(c, d, t, s, float(rest["tau"]), nsteps=18)
    torch.cuda.synchronize()
    assert torch.equal(a, d)
