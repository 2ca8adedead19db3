"""Helpers of the GPU tests: host <-> device copies of population fields."""
import numpy as np


def to_dev(a, dev, plane_stride=0):
    import torch
    a = np.ascontiguousarray(a, dtype=np.float32)
    q = a.shape[0]
    n = a[0].size
    ps = plane_stride or n
    buf = torch.zeros(q * ps, dtype=torch.float32, device=dev)
    buf.view(q, ps)[:, :n].copy_(torch.from_numpy(a.reshape(q, n)))
    return buf, ps


def from_dev(buf, shape, ps=None):
    q = shape[0]
    n = int(np.prod(shape[1:]))
    ps = ps or n
    return buf.view(q, ps)[:, :n].cpu().numpy().reshape(shape).astype(np.float64)


def bf16_to_np(t):
    """BF16 device tensor -> float64 numpy."""
    import torch
    return t.to(torch.float32).cpu().numpy().astype(np.float64)


def rel_l2(a, b):
    return float(np.sqrt(np.sum((a - b) ** 2) / max(np.sum(b ** 2), 1e-300)))
