"""Argument marshalling of the Python binding: device-buffer arguments must
be contiguous CUDA tensors of the right dtype and size (a host tensor would
hand a kernel a host address), host-buffer arguments CPU tensors or arrays.
Every check raises ValueError before the library is called.  The CPU part
runs without a GPU; the CUDA-tensor part is marked gpu."""
import numpy as np
import pytest

from paper_2504_14494_gb300 import lib as L


def test_host_tensors_are_rejected_for_device_arguments(lbmlib):
    torch = pytest.importorskip("torch")
    s = L.shape(8, 8)
    f = torch.zeros(9 * 64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        L.lbm_step_bgk(f, f, None, s, 0.8)
    with pytest.raises(ValueError, match="CUDA tensor"):
        L.lbm_init_tgv(np.zeros(9 * 64, np.float32), s, 1.0, 0.01, 0.1, 0.1)
    with pytest.raises(ValueError, match="CUDA tensor"):
        L.gnn_pack(torch.zeros(L.gnn_param_count()), None)
    with pytest.raises(ValueError, match="CUDA tensor"):
        L.lbm_moments(None, s, rho=torch.zeros(64))
    # raw integer addresses and None still reach the library (NULL -> LBM_ERR_ARG)
    with pytest.raises(L.LbmError) as e:
        L.lbm_step_bgk(None, None, None, s, 0.8, stream=0)
    assert e.value.code == L.LBM_ERR_ARG


def test_host_arguments_are_checked(lbmlib):
    torch = pytest.importorskip("torch")
    s = L.shape(4, 4)
    with pytest.raises(ValueError, match="dtype"):
        L.lbm_step_bgk_host(torch.zeros(9 * 16, dtype=torch.float64), None, s, 0.8)
    with pytest.raises(ValueError, match="elements"):
        L.lbm_step_bgk_host(torch.zeros(9 * 16 - 1), None, s, 0.8)
    with pytest.raises(ValueError, match="elements"):
        L.lbm_step_bgk_host(torch.zeros(9 * 16), None, s, 0.8,
                            totals_host=torch.zeros(4, dtype=torch.float64))
    with pytest.raises(ValueError, match="contiguous"):
        L.lbm_step_bgk_host(torch.zeros(2 * 9 * 16)[::2], None, s, 0.8)
    with pytest.raises(ValueError, match="dtype"):
        L.gnn_params_init_xavier(torch.zeros(L.gnn_param_count(), dtype=torch.float64), 0)


@pytest.mark.gpu
def test_cuda_tensors_are_checked(lbmlib, cuda):
    import torch
    s = L.shape(16, 8, 2, 300)  # plane stride 300: buffers span 8 * 300 + 256 values
    good = torch.zeros(8 * 300 + 256, device=cuda)
    with pytest.raises(ValueError, match="elements"):
        L.lbm_step_bgk(good, torch.zeros(9 * 256, device=cuda), None, s, 0.8)
    with pytest.raises(ValueError, match="dtype"):
        L.lbm_step_bgk(good, good.double(), None, s, 0.8)
    with pytest.raises(ValueError, match="contiguous"):
        L.lbm_step_bgk(good, torch.zeros(2 * good.numel(), device=cuda)[::2], None, s, 0.8)
    with pytest.raises(ValueError, match="taus"):
        L.lbm_step_bgk(good, torch.zeros_like(good), None, s, 0.8,
                       taus=torch.full((1,), 0.8, device=cuda))
    with pytest.raises(ValueError, match="bytes"):
        L.gnn_pack(torch.zeros(L.gnn_param_count(), device=cuda),
                   torch.zeros(16, dtype=torch.uint8, device=cuda))
    out = torch.zeros_like(good)
    L.lbm_step_bgk(good + 1.0 / 9, out, None, s, 0.8)  # valid arguments still run
    assert L.lbm_get_status() == L.LBM_OK
