"""Thin ctypes binding of liblbmgnn.so (argument marshalling only).

Every function here has the name and argument order of the C entry point in
include/lbmgnn.h.  Buffer arguments accept a torch tensor (its data_ptr() is
passed), a raw integer address (trusted), or None for a NULL pointer.  A
tensor for a device buffer must be a contiguous CUDA tensor of the dtype and
at least the size the call implies (dptr), one for a host buffer a CPU
tensor or numpy array (hptr); otherwise ValueError is raised before the
library is called.  `stream` defaults to torch's current CUDA stream.  A
non-zero status raises LbmError.

There is no fallback: if the shared library is missing or cannot be loaded,
every call raises.
"""
import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "liblbmgnn.so")

_lib = None


class LbmError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})" if what else
                         f"{status_string(code)} ({code})")


class lbm_shape(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nb", ctypes.c_int32),
                ("plane_stride", ctypes.c_int64)]


def shape(nx, ny, nb=1, plane_stride=0):
    return lbm_shape(int(nx), int(ny), int(nb), int(plane_stride))


class lbm_lattice_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("collision", ctypes.c_int32),
                ("tau", ctypes.c_float)]


LBM_COLLIDE_BGK, LBM_COLLIDE_GNN = 0, 1
# status codes (include/lbmgnn.h)
(LBM_OK, LBM_ERR_ARG, LBM_ERR_ALIAS, LBM_ERR_SIZE, LBM_ERR_TAU, LBM_ERR_BLOB, LBM_ERR_CUDA,
 LBM_ERR_NONFINITE, LBM_ERR_TIMEOUT, LBM_ERR_BOUNDS, LBM_ERR_WORKSPACE) = range(0, -11, -1)


_VP = ctypes.c_void_p
_SIGS = {
    "lbm_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "lbm_version": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "lbm_get_status": (ctypes.c_int, [_VP]),
    "lbm_selftest_wait_timeout": (ctypes.c_int, [ctypes.c_longlong, _VP]),
    "lbm_init_tgv": (ctypes.c_int, [_VP, lbm_shape, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int, _VP]),
    "lbm_step_bgk": (ctypes.c_int, [_VP, _VP, _VP, lbm_shape, ctypes.c_float, _VP, ctypes.c_int,
                                    _VP, _VP]),
    "lbm_moments": (ctypes.c_int, [_VP, lbm_shape, _VP, _VP, _VP, _VP, _VP]),
    "lbm_host_workspace_bytes": (ctypes.c_size_t, [lbm_shape]),
    "lbm_step_bgk_host": (ctypes.c_int, [_VP, _VP, lbm_shape, ctypes.c_float, _VP, ctypes.c_int,
                                         _VP, _VP, ctypes.c_size_t, _VP]),
    "lbm_step_channel": (ctypes.c_int, [_VP, _VP, _VP, lbm_shape, ctypes.c_float, _VP,
                                        ctypes.c_float, ctypes.c_int, _VP, _VP]),
    "gnn_param_count": (ctypes.c_size_t, []),
    "gnn_trainable_count": (ctypes.c_size_t, []),
    "gnn_params_init_xavier": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_float, ctypes.c_int]),
    "gnn_packed_bytes": (ctypes.c_size_t, []),
    "gnn_pack": (ctypes.c_int, [_VP, _VP, _VP]),
    "gnn_step_workspace_bytes": (ctypes.c_size_t, [lbm_shape]),
    "lbm_step_gnn": (ctypes.c_int, [_VP, _VP, lbm_shape, ctypes.c_float, _VP, _VP, _VP, _VP,
                                    ctypes.c_size_t, _VP]),
    "gnn_saved_bytes": (ctypes.c_size_t, [lbm_shape]),
    "gnn_forward": (ctypes.c_int, [_VP, lbm_shape, _VP, _VP, _VP, _VP]),
    "lbm_stream": (ctypes.c_int, [_VP, _VP, lbm_shape, _VP]),
    "lbm_init_tgv_batch": (ctypes.c_int, [_VP, lbm_shape, _VP, ctypes.c_int, _VP]),
    "lbm_restrict": (ctypes.c_int, [_VP, lbm_shape, _VP, lbm_shape, ctypes.c_int, ctypes.c_float,
                                    _VP, ctypes.c_float, _VP, _VP]),
    "gnn_loss_workspace_bytes": (ctypes.c_size_t, [lbm_shape]),
    "gnn_collide_loss": (ctypes.c_int, [_VP, _VP, _VP, lbm_shape, ctypes.c_float, _VP, _VP, _VP,
                                        _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "gnn_backward_workspace_bytes": (ctypes.c_size_t, [lbm_shape]),
    "gnn_backward": (ctypes.c_int, [_VP, lbm_shape, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_size_t,
                                    _VP]),
    "gnn_adamw": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int64, ctypes.c_float,
                                 ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                 _VP]),
    "gnn_train_workspace_bytes": (ctypes.c_size_t, [lbm_shape]),
    "gnn_train_step": (ctypes.c_int, [_VP, _VP, lbm_shape, ctypes.c_float, _VP, _VP, _VP, _VP, _VP,
                                      ctypes.c_int64, ctypes.c_float, ctypes.c_float, _VP, _VP,
                                      _VP, ctypes.c_size_t, _VP]),
    "lbm_step_gnn_noalloc": (ctypes.c_int, [_VP, _VP, lbm_shape, ctypes.c_float, _VP, _VP, _VP,
                                            _VP]),
    "lbm_step_gnn_mlp": (ctypes.c_int, [_VP, _VP, lbm_shape, ctypes.c_float, _VP, _VP, _VP, _VP]),
    "gnn_channel_workspace_bytes": (ctypes.c_size_t, [lbm_shape]),
    "lbm_step_gnn_channel": (ctypes.c_int, [_VP, _VP, lbm_shape, ctypes.c_float, _VP,
                                            ctypes.c_float, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "lbm_pair_weights_workspace_bytes": (ctypes.c_size_t, [lbm_shape]),
    "lbm_pair_weights": (ctypes.c_int, [_VP, _VP, lbm_shape, ctypes.c_float, _VP, _VP, _VP,
                                        ctypes.c_size_t, _VP]),
    "gnn_train_step_weighted": (ctypes.c_int, [_VP, _VP, lbm_shape, ctypes.c_float, _VP, _VP, _VP,
                                               _VP, _VP, _VP, ctypes.c_int64, ctypes.c_float,
                                               ctypes.c_float, _VP, _VP, _VP, ctypes.c_size_t,
                                               _VP]),
    "gnn_rollout_workspace_bytes": (ctypes.c_size_t, [lbm_shape, ctypes.c_int]),
    "gnn_train_step_rollout": (ctypes.c_int, [_VP, _VP, ctypes.c_int, lbm_shape, ctypes.c_float,
                                              _VP, _VP, _VP, _VP, _VP, ctypes.c_int64,
                                              ctypes.c_float, ctypes.c_float, _VP, _VP, _VP,
                                              ctypes.c_size_t, _VP]),
    "lbm_restrict_channel": (ctypes.c_int, [_VP, lbm_shape, _VP, lbm_shape, ctypes.c_int,
                                            ctypes.c_float, _VP, ctypes.c_float, _VP,
                                            ctypes.c_float, _VP, _VP]),
    "gnn_train_step_channel": (ctypes.c_int, [_VP, _VP, lbm_shape, ctypes.c_float, _VP,
                                              ctypes.c_float, _VP, _VP, _VP, _VP, _VP, _VP,
                                              ctypes.c_int64, ctypes.c_float, ctypes.c_float, _VP,
                                              _VP, _VP, ctypes.c_size_t, _VP]),
    "lbm_batch_plan_create": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "lbm_batch_plan_destroy": (None, [_VP]),
    "lbm_batch_nodes": (ctypes.c_int64, [_VP]),
    "lbm_batch_offsets": (ctypes.c_int, [_VP, _VP]),
    "lbm_batch_workspace_bytes": (ctypes.c_size_t, [_VP]),
    "lbm_batch_init_tgv": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
    "lbm_batch_run": (ctypes.c_int, [_VP, _VP, _VP, _VP, ctypes.c_int, _VP, _VP, ctypes.c_size_t,
                                     _VP]),
    "lbm_autotune_save": (ctypes.c_int, [ctypes.c_char_p]),
    "lbm_autotune_load": (ctypes.c_int, [ctypes.c_char_p]),
}

# Largest lattice (nb*ny*nx nodes) lbm_step_gnn_noalloc accepts (include/lbmgnn.h).
LBM_STEP_GNN_NOALLOC_MAX_NODES = 32768


def load(path=None):
    """Load the shared library (once).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with "
                           "paper_2504_14494_gb300.build.build() (no CPU fallback exists)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names bound by this module (each must be exported by the library)."""
    return list(_SIGS)


def register(name, restype, argtypes):
    """Declare one more entry point (used by the other binding modules)."""
    _SIGS[name] = (restype, argtypes)
    if _lib is not None:
        fn = getattr(_lib, name)
        fn.restype = restype
        fn.argtypes = argtypes


def _torch():
    import torch
    return torch


def _elems(s):
    """(nodes, plane stride, elements a population buffer of shape s spans)."""
    n = int(s.nx) * int(s.ny) * int(s.nb)
    ps = int(s.plane_stride) or n
    return n, ps, 8 * ps + n


def dptr(x, name, dtype=None, numel=0, nbytes_min=0):
    """Address of a DEVICE buffer argument: a contiguous CUDA tensor (of
    `dtype`, with at least `numel` elements and `nbytes_min` bytes when
    given), a raw int address (trusted), or None (NULL).  Anything else
    raises ValueError before the library is called: a host tensor here would
    hand a kernel a host address."""
    if x is None or isinstance(x, int):
        return x
    torch = _torch()
    if not isinstance(x, torch.Tensor):
        raise ValueError(f"{name}: a CUDA tensor or a device address is required, "
                         f"not {type(x).__name__}")
    if not x.is_cuda:
        raise ValueError(f"{name}: a CUDA tensor is required (got one on {x.device})")
    return _checked_tensor(x, name, dtype, numel, nbytes_min)


def hptr(x, name, dtype=None, numel=0):
    """Address of a HOST buffer argument: a contiguous CPU tensor or numpy
    array (of `dtype` and at least `numel` elements when given), a raw int
    address, or None."""
    if x is None or isinstance(x, int):
        return x
    import numpy as np
    if isinstance(x, np.ndarray):
        x = _torch().from_numpy(x)
    torch = _torch()
    if not isinstance(x, torch.Tensor) or x.is_cuda:
        raise ValueError(f"{name}: a host (CPU) tensor or array is required")
    return _checked_tensor(x, name, dtype, numel, 0)


def _checked_tensor(x, name, dtype, numel, nbytes_min):
    if not x.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if dtype is not None and x.dtype != dtype:
        raise ValueError(f"{name}: dtype {x.dtype}, {dtype} required")
    if x.numel() < numel:
        raise ValueError(f"{name}: {x.numel()} elements, at least {numel} required")
    if x.numel() * x.element_size() < nbytes_min:
        raise ValueError(f"{name}: {x.numel() * x.element_size()} bytes, at least "
                         f"{nbytes_min} required")
    return x.data_ptr()


def _f32():
    return _torch().float32


def _f64():
    return _torch().float64


def stream_ptr(stream=None):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def check(rc, what=""):
    if rc != 0:
        raise LbmError(rc, what)
    return rc


def status_string(code):
    return load().lbm_status_string(int(code)).decode()


def lbm_version():
    """(ABI version, packed-parameter layout version) of the loaded library."""
    abi, layout = ctypes.c_int(0), ctypes.c_int(0)
    check(load().lbm_version(ctypes.byref(abi), ctypes.byref(layout)), "lbm_version")
    return abi.value, layout.value


# --- BGK path ------------------------------------------------------------------------
def lbm_get_status(stream=None):
    """Synchronise the stream and return (not raise) the device status code."""
    return load().lbm_get_status(stream_ptr(stream))


def lbm_selftest_wait_timeout(max_cycles, stream=None):
    check(load().lbm_selftest_wait_timeout(int(max_cycles), stream_ptr(stream)),
          "lbm_selftest_wait_timeout")


def lbm_init_tgv(f, s, rho0, u0, kx, ky, pressure_consistent=False, stream=None):
    _, _, fe = _elems(s)
    check(load().lbm_init_tgv(dptr(f, "f", _f32(), fe), s, rho0, u0, kx, ky,
                              int(bool(pressure_consistent)), stream_ptr(stream)), "lbm_init_tgv")


def lbm_step_bgk(f_in, f_out, f_tmp, s, tau, taus=None, nsteps=1, totals=None, stream=None):
    _, _, fe = _elems(s)
    f32 = _f32()
    check(load().lbm_step_bgk(dptr(f_in, "f_in", f32, fe), dptr(f_out, "f_out", f32, fe),
                              dptr(f_tmp, "f_tmp", f32, fe), s, float(tau),
                              dptr(taus, "taus", f32, int(s.nb)), int(nsteps),
                              dptr(totals, "totals", _f64(), 5), stream_ptr(stream)),
          "lbm_step_bgk")


def lbm_step_channel(f_in, f_out, f_tmp, s, tau, taus=None, force_x=0.0, nsteps=1, totals=None,
                     stream=None):
    _, _, fe = _elems(s)
    f32 = _f32()
    check(load().lbm_step_channel(dptr(f_in, "f_in", f32, fe), dptr(f_out, "f_out", f32, fe),
                                  dptr(f_tmp, "f_tmp", f32, fe), s, float(tau),
                                  dptr(taus, "taus", f32, int(s.nb)), float(force_x), int(nsteps),
                                  dptr(totals, "totals", _f64(), 5), stream_ptr(stream)),
          "lbm_step_channel")


def lbm_moments(f, s, rho=None, ux=None, uy=None, totals=None, stream=None):
    n, _, fe = _elems(s)
    f32 = _f32()
    check(load().lbm_moments(dptr(f, "f", f32, fe), s, dptr(rho, "rho", f32, n),
                             dptr(ux, "ux", f32, n), dptr(uy, "uy", f32, n),
                             dptr(totals, "totals", _f64(), 5), stream_ptr(stream)), "lbm_moments")


def lbm_host_workspace_bytes(s):
    return load().lbm_host_workspace_bytes(s)


def lbm_step_bgk_host(f_in_host, f_out_host, s, tau, taus_host=None, nsteps=1,
                      totals_host=None, workspace=None, ws_bytes=None, stream=None):
    """lbm_step_bgk on a state in host memory (CPU tensors, page-locked for
    overlap); asynchronous on `stream` (see include/lbmgnn.h)."""
    _, _, fe = _elems(s)
    f32 = _f32()
    check(load().lbm_step_bgk_host(hptr(f_in_host, "f_in_host", f32, fe),
                                   hptr(f_out_host, "f_out_host", f32, fe), s, float(tau),
                                   hptr(taus_host, "taus_host", f32, int(s.nb)), int(nsteps),
                                   hptr(totals_host, "totals_host", _f64(), 5),
                                   dptr(workspace, "workspace"),
                                   int(nbytes(workspace) if ws_bytes is None else ws_bytes),
                                   stream_ptr(stream)), "lbm_step_bgk_host")


# --- GNN path ------------------------------------------------------------------------
def gnn_params_init_xavier(params_host, seed, s_df=1e-4, variant=0):
    """Fills a host float32 array / CPU tensor of gnn_param_count() values
    (see include/lbmgnn.h); returns it."""
    import numpy as np
    if isinstance(params_host, np.ndarray):
        if params_host.dtype != np.float32 or not params_host.flags.c_contiguous:
            raise ValueError("params_host must be a contiguous float32 array")
        addr = params_host.ctypes.data
    else:
        addr = hptr(params_host, "params_host", _f32(), gnn_param_count())
    check(load().gnn_params_init_xavier(addr, int(seed), float(s_df), int(variant)),
          "gnn_params_init_xavier")
    return params_host


def gnn_param_count():
    return load().gnn_param_count()


def gnn_trainable_count():
    return load().gnn_trainable_count()


def gnn_packed_bytes():
    return load().gnn_packed_bytes()


def gnn_pack(params, packed, stream=None):
    check(load().gnn_pack(dptr(params, "params", _f32(), gnn_param_count()),
                          dptr(packed, "packed", nbytes_min=gnn_packed_bytes()),
                          stream_ptr(stream)), "gnn_pack")


def gnn_step_workspace_bytes(s):
    return load().gnn_step_workspace_bytes(s)


def nbytes(t):
    return 0 if t is None else t.numel() * t.element_size()


def lbm_step_gnn(f_in, f_out, s, tau, taus, packed, totals, workspace, ws_bytes=None,
                 stream=None):
    if ws_bytes is None:
        ws_bytes = nbytes(workspace)
    _, _, fe = _elems(s)
    f32 = _f32()
    check(load().lbm_step_gnn(dptr(f_in, "f_in", f32, fe), dptr(f_out, "f_out", f32, fe), s,
                              float(tau), dptr(taus, "taus", f32, int(s.nb)),
                              dptr(packed, "packed", nbytes_min=gnn_packed_bytes()),
                              dptr(totals, "totals", _f64(), 5), dptr(workspace, "workspace"),
                              int(ws_bytes), stream_ptr(stream)), "lbm_step_gnn")


def lbm_step_gnn_mlp(f_in, f_out, s, tau, taus, packed, totals, stream=None):
    """The paper's Fig. 2 (MLP-only) network's GNN-LBM step as one fused
    kernel, no workspace (see include/lbmgnn.h)."""
    _, _, fe = _elems(s)
    f32 = _f32()
    check(load().lbm_step_gnn_mlp(dptr(f_in, "f_in", f32, fe), dptr(f_out, "f_out", f32, fe), s,
                                  float(tau), dptr(taus, "taus", f32, int(s.nb)),
                                  dptr(packed, "packed", nbytes_min=gnn_packed_bytes()),
                                  dptr(totals, "totals", _f64(), 5), stream_ptr(stream)),
          "lbm_step_gnn_mlp")


def gnn_channel_workspace_bytes(s):
    return load().gnn_channel_workspace_bytes(s)


def lbm_step_gnn_channel(f_in, f_out, s, tau, taus, force_x, packed, totals, workspace,
                         ws_bytes=None, stream=None):
    """GNN-LBM step of the channel (walls, Guo forcing, Eq. 3; see
    include/lbmgnn.h)."""
    if ws_bytes is None:
        ws_bytes = nbytes(workspace)
    _, _, fe = _elems(s)
    f32 = _f32()
    check(load().lbm_step_gnn_channel(dptr(f_in, "f_in", f32, fe), dptr(f_out, "f_out", f32, fe),
                                      s, float(tau), dptr(taus, "taus", f32, int(s.nb)),
                                      float(force_x),
                                      dptr(packed, "packed", nbytes_min=gnn_packed_bytes()),
                                      dptr(totals, "totals", _f64(), 5),
                                      dptr(workspace, "workspace"), int(ws_bytes),
                                      stream_ptr(stream)), "lbm_step_gnn_channel")


def gnn_saved_bytes(s):
    return load().gnn_saved_bytes(s)


def gnn_forward(f_pre, s, packed, saved, y, stream=None):
    n, _, fe = _elems(s)
    check(load().gnn_forward(dptr(f_pre, "f_pre", _f32(), fe), s,
                             dptr(packed, "packed", nbytes_min=gnn_packed_bytes()),
                             dptr(saved, "saved", nbytes_min=gnn_saved_bytes(s)),
                             dptr(y, "y", _f32(), 10 * n), stream_ptr(stream)), "gnn_forward")


# --- auxiliary lattice operations and training ------------------------------------
def lbm_stream(f_in, f_out, s, stream=None):
    _, _, fe = _elems(s)
    check(load().lbm_stream(dptr(f_in, "f_in", _f32(), fe), dptr(f_out, "f_out", _f32(), fe), s,
                            stream_ptr(stream)), "lbm_stream")


def lbm_init_tgv_batch(f, s, params, pressure_consistent=False, stream=None):
    _, _, fe = _elems(s)
    check(load().lbm_init_tgv_batch(dptr(f, "f", _f32(), fe), s,
                                    dptr(params, "params", _f64(), 4 * int(s.nb)),
                                    int(bool(pressure_consistent)), stream_ptr(stream)),
          "lbm_init_tgv_batch")


def lbm_restrict(f_fine, fine, f_coarse, coarse, factor, tau_f, taus_f, tau_c, taus_c,
                 stream=None):
    f32 = _f32()
    check(load().lbm_restrict(dptr(f_fine, "f_fine", f32, _elems(fine)[2]), fine,
                              dptr(f_coarse, "f_coarse", f32, _elems(coarse)[2]), coarse,
                              int(factor), float(tau_f), dptr(taus_f, "taus_f", f32, int(fine.nb)),
                              float(tau_c), dptr(taus_c, "taus_c", f32, int(coarse.nb)),
                              stream_ptr(stream)), "lbm_restrict")


def lbm_restrict_channel(f_fine, fine, f_coarse, coarse, factor, tau_f, taus_f, tau_c, taus_c,
                         force_x_f, forces_x_f=None, stream=None):
    f32 = _f32()
    check(load().lbm_restrict_channel(
        dptr(f_fine, "f_fine", f32, _elems(fine)[2]), fine,
        dptr(f_coarse, "f_coarse", f32, _elems(coarse)[2]), coarse, int(factor), float(tau_f),
        dptr(taus_f, "taus_f", f32, int(fine.nb)), float(tau_c),
        dptr(taus_c, "taus_c", f32, int(coarse.nb)), float(force_x_f),
        dptr(forces_x_f, "forces_x_f", f32, int(fine.nb)), stream_ptr(stream)),
        "lbm_restrict_channel")


def gnn_loss_workspace_bytes(s):
    return load().gnn_loss_workspace_bytes(s)


def gnn_collide_loss(f_pre, y, f_target, s, tau, taus, packed, loss, dy, f_pred, workspace,
                     ws_bytes=None, stream=None):
    n, _, fe = _elems(s)
    f32 = _f32()
    check(load().gnn_collide_loss(dptr(f_pre, "f_pre", f32, fe), dptr(y, "y", f32, 10 * n),
                                  dptr(f_target, "f_target", f32, fe), s, float(tau),
                                  dptr(taus, "taus", f32, int(s.nb)),
                                  dptr(packed, "packed", nbytes_min=gnn_packed_bytes()),
                                  dptr(loss, "loss", _f64(), 1), dptr(dy, "dy", f32, 10 * n),
                                  dptr(f_pred, "f_pred", f32, fe), dptr(workspace, "workspace"),
                                  int(nbytes(workspace) if ws_bytes is None else ws_bytes),
                                  stream_ptr(stream)), "gnn_collide_loss")


def gnn_backward_workspace_bytes(s):
    return load().gnn_backward_workspace_bytes(s)


def gnn_backward(f_pre, s, packed, saved, dy, dparams, df_pre, workspace, ws_bytes=None,
                 stream=None):
    n, _, fe = _elems(s)
    f32 = _f32()
    check(load().gnn_backward(dptr(f_pre, "f_pre", f32, fe), s,
                              dptr(packed, "packed", nbytes_min=gnn_packed_bytes()),
                              dptr(saved, "saved", nbytes_min=gnn_saved_bytes(s)),
                              dptr(dy, "dy", f32, 10 * n),
                              dptr(dparams, "dparams", f32, gnn_trainable_count()),
                              dptr(df_pre, "df_pre", f32, fe), dptr(workspace, "workspace"),
                              int(nbytes(workspace) if ws_bytes is None else ws_bytes),
                              stream_ptr(stream)), "gnn_backward")


def gnn_adamw(params, grads, m, v, step, lr, wd, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    nt, f32 = gnn_trainable_count(), _f32()
    check(load().gnn_adamw(dptr(params, "params", f32, nt), dptr(grads, "grads", f32, nt),
                           dptr(m, "m", f32, nt), dptr(v, "v", f32, nt), int(step), float(lr),
                           float(wd), float(beta1), float(beta2), float(eps), stream_ptr(stream)),
          "gnn_adamw")


def gnn_train_workspace_bytes(s):
    return load().gnn_train_workspace_bytes(s)


def lbm_pair_weights_workspace_bytes(s):
    return load().lbm_pair_weights_workspace_bytes(s)


def lbm_pair_weights(f_in, f_target, s, tau, taus, weights, workspace, ws_bytes=None,
                     stream=None):
    """Per-lattice loss weights mean(D) / D_b from the one-step BGK residuals
    (see include/lbmgnn.h); weights: device FP32 [nb]."""
    _, _, fe = _elems(s)
    f32 = _f32()
    check(load().lbm_pair_weights(dptr(f_in, "f_in", f32, fe), dptr(f_target, "f_target", f32, fe),
                                  s, float(tau), dptr(taus, "taus", f32, int(s.nb)),
                                  dptr(weights, "weights", f32, int(s.nb)),
                                  dptr(workspace, "workspace"),
                                  int(nbytes(workspace) if ws_bytes is None else ws_bytes),
                                  stream_ptr(stream)), "lbm_pair_weights")


def gnn_train_step_weighted(f_in, f_target, s, tau, taus, lat_weights, params, packed, adam_m,
                            adam_v, step, lr, wd, loss, grads, workspace, ws_bytes=None,
                            stream=None):
    _, _, fe = _elems(s)
    nt, f32 = gnn_trainable_count(), _f32()
    check(load().gnn_train_step_weighted(
        dptr(f_in, "f_in", f32, fe), dptr(f_target, "f_target", f32, fe), s, float(tau),
        dptr(taus, "taus", f32, int(s.nb)), dptr(lat_weights, "lat_weights", f32, int(s.nb)),
        dptr(params, "params", f32, gnn_param_count()),
        dptr(packed, "packed", nbytes_min=gnn_packed_bytes()),
        dptr(adam_m, "adam_m", f32, nt), dptr(adam_v, "adam_v", f32, nt), int(step), float(lr),
        float(wd), dptr(loss, "loss", _f64(), 1), dptr(grads, "grads", f32, nt),
        dptr(workspace, "workspace"), int(nbytes(workspace) if ws_bytes is None else ws_bytes),
        stream_ptr(stream)), "gnn_train_step_weighted")


def gnn_rollout_workspace_bytes(s, K):
    return int(load().gnn_rollout_workspace_bytes(s, int(K)))


def gnn_train_step_rollout(f_in, f_targets, K, s, tau, taus, params, packed, adam_m, adam_v, step,
                           lr, wd, loss, grads, workspace, ws_bytes=None, stream=None):
    _, _, fe = _elems(s)
    ps = int(s.plane_stride) or int(s.nx) * int(s.ny) * int(s.nb)
    nt, f32 = gnn_trainable_count(), _f32()
    check(load().gnn_train_step_rollout(
        dptr(f_in, "f_in", f32, fe), dptr(f_targets, "f_targets", f32, (int(K) - 1) * 9 * ps + fe),
        int(K), s, float(tau), dptr(taus, "taus", f32, int(s.nb)),
        dptr(params, "params", f32, gnn_param_count()),
        dptr(packed, "packed", nbytes_min=gnn_packed_bytes()),
        dptr(adam_m, "adam_m", f32, nt), dptr(adam_v, "adam_v", f32, nt), int(step), float(lr),
        float(wd), dptr(loss, "loss", _f64(), 1), dptr(grads, "grads", f32, nt),
        dptr(workspace, "workspace"), int(nbytes(workspace) if ws_bytes is None else ws_bytes),
        stream_ptr(stream)), "gnn_train_step_rollout")


def gnn_train_step_channel(f_in, f_target, s, tau, taus, force_x, forces_x, lat_weights, params,
                           packed, adam_m, adam_v, step, lr, wd, loss, grads, workspace,
                           ws_bytes=None, stream=None):
    _, _, fe = _elems(s)
    nt, f32 = gnn_trainable_count(), _f32()
    check(load().gnn_train_step_channel(
        dptr(f_in, "f_in", f32, fe), dptr(f_target, "f_target", f32, fe), s, float(tau),
        dptr(taus, "taus", f32, int(s.nb)), float(force_x),
        dptr(forces_x, "forces_x", f32, int(s.nb)),
        dptr(lat_weights, "lat_weights", f32, int(s.nb)),
        dptr(params, "params", f32, gnn_param_count()),
        dptr(packed, "packed", nbytes_min=gnn_packed_bytes()),
        dptr(adam_m, "adam_m", f32, nt), dptr(adam_v, "adam_v", f32, nt), int(step), float(lr),
        float(wd), dptr(loss, "loss", _f64(), 1), dptr(grads, "grads", f32, nt),
        dptr(workspace, "workspace"), int(nbytes(workspace) if ws_bytes is None else ws_bytes),
        stream_ptr(stream)), "gnn_train_step_channel")


def gnn_train_step(f_in, f_target, s, tau, taus, params, packed, adam_m, adam_v, step, lr, wd,
                   loss, grads, workspace, ws_bytes=None, stream=None):
    _, _, fe = _elems(s)
    nt, f32 = gnn_trainable_count(), _f32()
    check(load().gnn_train_step(dptr(f_in, "f_in", f32, fe), dptr(f_target, "f_target", f32, fe),
                                s, float(tau), dptr(taus, "taus", f32, int(s.nb)),
                                dptr(params, "params", f32, gnn_param_count()),
                                dptr(packed, "packed", nbytes_min=gnn_packed_bytes()),
                                dptr(adam_m, "adam_m", f32, nt), dptr(adam_v, "adam_v", f32, nt),
                                int(step), float(lr), float(wd), dptr(loss, "loss", _f64(), 1),
                                dptr(grads, "grads", f32, nt), dptr(workspace, "workspace"),
                                int(nbytes(workspace) if ws_bytes is None else ws_bytes),
                                stream_ptr(stream)), "gnn_train_step")


def lbm_step_gnn_noalloc(f_in, f_out, s, tau, taus, packed, totals, stream=None):
    """lbm_step_gnn with the library's fixed internal scratch (no workspace
    argument, nothing allocated; see include/lbmgnn.h)."""
    _, _, fe = _elems(s)
    f32 = _f32()
    check(load().lbm_step_gnn_noalloc(dptr(f_in, "f_in", f32, fe), dptr(f_out, "f_out", f32, fe),
                                      s, float(tau), dptr(taus, "taus", f32, int(s.nb)),
                                      dptr(packed, "packed", nbytes_min=gnn_packed_bytes()),
                                      dptr(totals, "totals", _f64(), 5), stream_ptr(stream)),
          "lbm_step_gnn_noalloc")


# --- batched runs -----------------------------------------------------------------------
def lbm_batch_plan_create(lattices):
    """lattices: iterable of (nx, ny, collision, tau).  Returns the plan handle."""
    lat = list(lattices)
    arr = (lbm_lattice_desc * len(lat))(*[lbm_lattice_desc(int(a), int(b), int(c), float(t))
                                           for a, b, c, t in lat])
    out = ctypes.c_void_p()
    check(load().lbm_batch_plan_create(ctypes.cast(arr, ctypes.c_void_p), len(lat),
                                       ctypes.byref(out)), "lbm_batch_plan_create")
    return out.value


def lbm_batch_plan_destroy(plan):
    load().lbm_batch_plan_destroy(plan)


def lbm_batch_nodes(plan):
    return load().lbm_batch_nodes(plan)


def lbm_batch_offsets(plan, n):
    import numpy as np
    out = np.zeros(n, dtype=np.int64)
    check(load().lbm_batch_offsets(plan, out.ctypes.data), "lbm_batch_offsets")
    return out


def lbm_batch_workspace_bytes(plan):
    return load().lbm_batch_workspace_bytes(plan)


def lbm_batch_init_tgv(plan, f, params, pressure_consistent=False, stream=None):
    """params: host float64 array [n][4] = (rho0, u0, kx, ky)."""
    import numpy as np
    prm = np.ascontiguousarray(params, dtype=np.float64)
    fe = 9 * max(lbm_batch_nodes(plan), 0) if plan else 0
    check(load().lbm_batch_init_tgv(plan, dptr(f, "f", _f32(), fe), prm.ctypes.data,
                                    int(bool(pressure_consistent)), stream_ptr(stream)),
          "lbm_batch_init_tgv")


def lbm_batch_run(plan, f_in, f_out, f_tmp, steps, packed, workspace, ws_bytes=None, stream=None):
    fe = 9 * max(lbm_batch_nodes(plan), 0) if plan else 0
    f32 = _f32()
    check(load().lbm_batch_run(plan, dptr(f_in, "f_in", f32, fe), dptr(f_out, "f_out", f32, fe),
                               dptr(f_tmp, "f_tmp", f32, fe), int(steps),
                               dptr(packed, "packed", nbytes_min=gnn_packed_bytes()),
                               dptr(workspace, "workspace"),
                               int(nbytes(workspace) if ws_bytes is None else ws_bytes),
                               stream_ptr(stream)), "lbm_batch_run")


def lbm_autotune_save(path):
    check(load().lbm_autotune_save(str(path).encode()), "lbm_autotune_save")


def lbm_autotune_load(path):
    check(load().lbm_autotune_load(str(path).encode()), "lbm_autotune_load")
