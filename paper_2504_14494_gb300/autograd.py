"""torch.autograd.Function around the hand-written CUDA forward and backward
of the network (gnn_forward / gnn_backward of liblbmgnn.so).

    y = GnnFunction.apply(f_pre, params, shape)

f_pre: pre-collision populations (device FP32, 9 planes of `shape`);
params: the FP32 parameter vector (38,948 values; the 26 fixed values get a
zero gradient).  Returns y as a [10, N] tensor (plane o = head output o).
The backward returns dL/df_pre and dL/dparams from the library's kernels.
"""
import torch

from . import lib as L


class GnnFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, f_pre, params, shape):
        n = shape.nx * shape.ny * shape.nb
        dev = f_pre.device
        packed = torch.empty(L.gnn_packed_bytes(), dtype=torch.uint8, device=dev)
        L.gnn_pack(params.detach(), packed)
        saved = torch.empty(L.gnn_saved_bytes(shape), dtype=torch.uint8, device=dev)
        y = torch.empty(10 * n, dtype=torch.float32, device=dev)
        L.gnn_forward(f_pre.detach(), shape, packed, saved, y)
        ctx.save_for_backward(f_pre)
        ctx.packed, ctx.saved, ctx.shape, ctx.nparams = packed, saved, shape, params.numel()
        return y.view(10, n)

    @staticmethod
    def backward(ctx, dy):
        (f_pre,) = ctx.saved_tensors
        dev = f_pre.device
        dparams = torch.zeros(ctx.nparams, dtype=torch.float32, device=dev)
        df = torch.empty_like(f_pre) if ctx.needs_input_grad[0] else None
        ws = torch.empty(L.gnn_backward_workspace_bytes(ctx.shape), dtype=torch.uint8, device=dev)
        L.gnn_backward(f_pre.detach(), ctx.shape, ctx.packed, ctx.saved,
                       dy.contiguous().view(-1), dparams, df, ws)
        return df, dparams, None
