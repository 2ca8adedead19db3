"""The hand-written CUDA backward behind torch.autograd.Function
(paper_2504_14494_gb300.autograd.GnnFunction), driven by torch's autograd.

Stated tolerances:
  * gradients of L = sum(w * y) with respect to the parameters and to
    f_pre against the FP64 oracle's hand-derived backward: per parameter
    tensor cosine >= 0.999 and relative L2 <= 3e-2 (as gnn_backward: BF16
    operands and activations, FP32 accumulation); the 26 fixed values
    (normaliser, s_df, variant) get exactly zero;
  * directional derivatives <grad, v> against central finite differences
    of the CUDA forward itself, Richardson-extrapolated from steps of 1 %
    and 0.5 % of every parameter (or population) moved, along directions
    with the gradient's signs (so that the derivative does not cancel):
    relative error <= 3e-2.  The FP64 oracle's own forward gives 0.07-0.3 %
    this way and 0.25-0.4 % with BF16-rounded weights; the CUDA forward
    (BF16 activations as well) gave 0.2-0.9 % on a GB300."""
import numpy as np
import pytest

from oracle import gnn, lbm
from paper_2504_14494_gb300 import inputs
from gpu_util import rel_l2

pytestmark = pytest.mark.gpu

NB, NY, NX = 2, 8, 12


def _f_pre(seed):
    f = lbm.tgv_init(NX, NY, 1.0, 0.06, 2 * np.pi / NX, 2 * np.pi / NY)
    f = np.stack([f * inputs.perturbation(f.shape, seed + b, 5e-2) for b in range(NB)], axis=1)
    return f.astype(np.float32)  # [9][NB][NY][NX]


def _setup(L, cuda, seed):
    import torch
    from paper_2504_14494_gb300.autograd import GnnFunction
    theta = inputs.xavier_params(seed, s_df=1e-2, bias_scale=0.1)
    f = _f_pre(seed)
    s = L.shape(NX, NY, NB)
    n = NB * NY * NX
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    w = torch.randn(10, n, generator=g, dtype=torch.float32).to(cuda)

    def loss(fd, p):  # summed in FP64, so that only the network's rounding reaches the quotients
        return (GnnFunction.apply(fd, p, s).double() * w.double()).sum()

    return theta, f, w, loss


def test_autograd_gradients_match_the_oracle(lbmlib, cuda):
    import torch
    theta, f, w, loss = _setup(lbmlib, cuda, 31)
    fd = torch.from_numpy(f.reshape(-1).copy()).to(cuda).requires_grad_()
    p = torch.from_numpy(theta.copy()).to(cuda).requires_grad_()
    loss(fd, p).backward()
    assert lbmlib.lbm_get_status() == 0
    gp = p.grad.double().cpu().numpy()
    gf = fd.grad.double().cpu().numpy().reshape(f.shape)
    assert np.all(gp[gnn.N_TRAINABLE:] == 0.0)
    pr = gnn.unpack(theta)
    per = NY * NX
    wn = w.double().cpu().numpy()
    g_ref = np.zeros(gnn.N_TRAINABLE)
    df_ref = np.zeros(f.shape)
    for b in range(NB):
        _, cache = gnn.forward(f[:, b].astype(np.float64), pr)
        gb, dfb = gnn.backward(wn[:, b * per:(b + 1) * per].T, cache, pr)
        g_ref += gnn.pack_grads(gb)
        df_ref[:, b] = dfb.reshape(9, NY, NX)
    o = 0
    for name, shape in gnn.SHAPES:
        k = int(np.prod(shape))
        a, r = gp[o:o + k], g_ref[o:o + k]
        o += k
        c = float(np.dot(a, r) / (np.linalg.norm(a) * np.linalg.norm(r) + 1e-300))
        assert c >= 0.999 and rel_l2(a, r) <= 3e-2, (name, c, rel_l2(a, r))
    assert rel_l2(gf, df_ref) <= 3e-2


def test_autograd_gradients_match_finite_differences(lbmlib, cuda):
    import torch
    theta, f, w, loss = _setup(lbmlib, cuda, 37)
    fd = torch.from_numpy(f.reshape(-1).copy()).to(cuda).requires_grad_()
    p = torch.from_numpy(theta.copy()).to(cuda).requires_grad_()
    loss(fd, p).backward()
    gp, gf = p.grad.double(), fd.grad.double()
    rng = np.random.default_rng(5)
    eps = 0.01

    def richardson(fn):
        d1 = (fn(eps) - fn(-eps)) / (2 * eps)
        d2 = (fn(eps / 2) - fn(-eps / 2)) / eps
        return (4 * d2 - d1) / 3

    with torch.no_grad():
        p0, f0 = p.detach(), fd.detach()
        for _ in range(2):  # parameters: each weight and bias moved by 0.5-1 x eps of itself
            r = np.sign(gp.cpu().numpy()) * rng.uniform(0.5, 1.0, theta.size)
            r[gnn.N_TRAINABLE:] = 0.0  # normaliser, s_df, variant stay fixed
            v = torch.from_numpy(r * np.abs(theta)).to(cuda)
            num = richardson(lambda e: loss(f0, (p0.double() + e * v).float()).double().item())
            ad = float((gp * v).sum())
            print(f"parameter direction: finite differences {num:.6e}, autograd {ad:.6e}")
            assert abs(num - ad) <= 3e-2 * abs(ad), (num, ad)
        for _ in range(2):  # populations
            u = np.sign(gf.cpu().numpy()) * rng.uniform(0.5, 1.0, f.size) * f.reshape(-1)
            ut = torch.from_numpy(u).to(cuda)
            num = richardson(lambda e: loss((f0.double() + e * ut).float(), p0).double().item())
            ad = float((gf * ut).sum())
            print(f"population direction: finite differences {num:.6e}, autograd {ad:.6e}")
            assert abs(num - ad) <= 3e-2 * abs(ad), (num, ad)
    assert lbmlib.lbm_get_status() == 0
