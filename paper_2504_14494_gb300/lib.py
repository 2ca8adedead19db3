"""Thin ctypes binding of liblbmgnn.so (argument marshalling only).

Every function here has the name and argument order of the C entry point in
include/lbmgnn.h.  Buffer arguments accept a torch tensor (its data_ptr() is
passed), a raw integer address, or None for a NULL pointer.  `stream`
defaults to torch's current CUDA stream.  A non-zero status raises LbmError.

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


def ptr(x):
    """Device/host address of a tensor, an int, or None (NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


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


# --- BGK path ------------------------------------------------------------------------
def lbm_get_status(stream=None):
    """Synchronise the stream and return (not raise) the device status code."""
    return load().lbm_get_status(stream_ptr(stream))


def lbm_selftest_wait_timeout(max_cycles, stream=None):
    check(load().lbm_selftest_wait_timeout(int(max_cycles), stream_ptr(stream)),
          "lbm_selftest_wait_timeout")


def lbm_init_tgv(f, s, rho0, u0, kx, ky, pressure_consistent=False, stream=None):
    check(load().lbm_init_tgv(ptr(f), s, rho0, u0, kx, ky, int(bool(pressure_consistent)),
                              stream_ptr(stream)), "lbm_init_tgv")


def lbm_step_bgk(f_in, f_out, f_tmp, s, tau, taus=None, nsteps=1, totals=None, stream=None):
    check(load().lbm_step_bgk(ptr(f_in), ptr(f_out), ptr(f_tmp), s, float(tau), ptr(taus),
                              int(nsteps), ptr(totals), stream_ptr(stream)), "lbm_step_bgk")


def lbm_step_channel(f_in, f_out, f_tmp, s, tau, taus=None, force_x=0.0, nsteps=1, totals=None,
                     stream=None):
    check(load().lbm_step_channel(ptr(f_in), ptr(f_out), ptr(f_tmp), s, float(tau), ptr(taus),
                                  float(force_x), int(nsteps), ptr(totals), stream_ptr(stream)),
          "lbm_step_channel")


def lbm_moments(f, s, rho=None, ux=None, uy=None, totals=None, stream=None):
    check(load().lbm_moments(ptr(f), s, ptr(rho), ptr(ux), ptr(uy), ptr(totals),
                             stream_ptr(stream)), "lbm_moments")


def lbm_host_workspace_bytes(s):
    return load().lbm_host_workspace_bytes(s)


def lbm_step_bgk_host(f_in_host, f_out_host, s, tau, taus_host=None, nsteps=1,
                      totals_host=None, workspace=None, ws_bytes=None, stream=None):
    """lbm_step_bgk on a state in host memory (CPU tensors, page-locked for
    overlap); asynchronous on `stream` (see include/lbmgnn.h)."""
    check(load().lbm_step_bgk_host(ptr(f_in_host), ptr(f_out_host), s, float(tau),
                                   ptr(taus_host), int(nsteps), ptr(totals_host), ptr(workspace),
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
        addr = ptr(params_host)
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
    check(load().gnn_pack(ptr(params), ptr(packed), stream_ptr(stream)), "gnn_pack")


def gnn_step_workspace_bytes(s):
    return load().gnn_step_workspace_bytes(s)


def nbytes(t):
    return 0 if t is None else t.numel() * t.element_size()


def lbm_step_gnn(f_in, f_out, s, tau, taus, packed, totals, workspace, ws_bytes=None,
                 stream=None):
    if ws_bytes is None:
        ws_bytes = nbytes(workspace)
    check(load().lbm_step_gnn(ptr(f_in), ptr(f_out), s, float(tau), ptr(taus), ptr(packed),
                              ptr(totals), ptr(workspace), int(ws_bytes), stream_ptr(stream)),
          "lbm_step_gnn")


def gnn_saved_bytes(s):
    return load().gnn_saved_bytes(s)


def gnn_forward(f_pre, s, packed, saved, y, stream=None):
    check(load().gnn_forward(ptr(f_pre), s, ptr(packed), ptr(saved), ptr(y), stream_ptr(stream)),
          "gnn_forward")


# --- auxiliary lattice operations and training ------------------------------------
def lbm_stream(f_in, f_out, s, stream=None):
    check(load().lbm_stream(ptr(f_in), ptr(f_out), s, stream_ptr(stream)), "lbm_stream")


def lbm_init_tgv_batch(f, s, params, pressure_consistent=False, stream=None):
    check(load().lbm_init_tgv_batch(ptr(f), s, ptr(params), int(bool(pressure_consistent)),
                                    stream_ptr(stream)), "lbm_init_tgv_batch")


def lbm_restrict(f_fine, fine, f_coarse, coarse, factor, tau_f, taus_f, tau_c, taus_c,
                 stream=None):
    check(load().lbm_restrict(ptr(f_fine), fine, ptr(f_coarse), coarse, int(factor), float(tau_f),
                              ptr(taus_f), float(tau_c), ptr(taus_c), stream_ptr(stream)),
          "lbm_restrict")


def gnn_loss_workspace_bytes(s):
    return load().gnn_loss_workspace_bytes(s)


def gnn_collide_loss(f_pre, y, f_target, s, tau, taus, packed, loss, dy, f_pred, workspace,
                     ws_bytes=None, stream=None):
    check(load().gnn_collide_loss(ptr(f_pre), ptr(y), ptr(f_target), s, float(tau), ptr(taus),
                                  ptr(packed), ptr(loss), ptr(dy), ptr(f_pred), ptr(workspace),
                                  int(nbytes(workspace) if ws_bytes is None else ws_bytes),
                                  stream_ptr(stream)), "gnn_collide_loss")


def gnn_backward_workspace_bytes(s):
    return load().gnn_backward_workspace_bytes(s)


def gnn_backward(f_pre, s, packed, saved, dy, dparams, df_pre, workspace, ws_bytes=None,
                 stream=None):
    check(load().gnn_backward(ptr(f_pre), s, ptr(packed), ptr(saved), ptr(dy), ptr(dparams),
                              ptr(df_pre), ptr(workspace),
                              int(nbytes(workspace) if ws_bytes is None else ws_bytes),
                              stream_ptr(stream)), "gnn_backward")


def gnn_adamw(params, grads, m, v, step, lr, wd, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    check(load().gnn_adamw(ptr(params), ptr(grads), ptr(m), ptr(v), int(step), float(lr),
                           float(wd), float(beta1), float(beta2), float(eps), stream_ptr(stream)),
          "gnn_adamw")


def gnn_train_workspace_bytes(s):
    return load().gnn_train_workspace_bytes(s)


def gnn_train_step(f_in, f_target, s, tau, taus, params, packed, adam_m, adam_v, step, lr, wd,
                   loss, grads, workspace, ws_bytes=None, stream=None):
    check(load().gnn_train_step(ptr(f_in), ptr(f_target), s, float(tau), ptr(taus), ptr(params),
                                ptr(packed), ptr(adam_m), ptr(adam_v), int(step), float(lr),
                                float(wd), ptr(loss), ptr(grads), ptr(workspace),
                                int(nbytes(workspace) if ws_bytes is None else ws_bytes),
                                stream_ptr(stream)), "gnn_train_step")


def lbm_step_gnn_noalloc(f_in, f_out, s, tau, taus, packed, totals, stream=None):
    """lbm_step_gnn with the library's fixed internal scratch (no workspace
    argument, nothing allocated; see include/lbmgnn.h)."""
    check(load().lbm_step_gnn_noalloc(ptr(f_in), ptr(f_out), s, float(tau), ptr(taus),
                                      ptr(packed), ptr(totals), stream_ptr(stream)),
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
    check(load().lbm_batch_init_tgv(plan, ptr(f), prm.ctypes.data, int(bool(pressure_consistent)),
                                    stream_ptr(stream)), "lbm_batch_init_tgv")


def lbm_batch_run(plan, f_in, f_out, f_tmp, steps, packed, workspace, ws_bytes=None, stream=None):
    check(load().lbm_batch_run(plan, ptr(f_in), ptr(f_out), ptr(f_tmp), int(steps), ptr(packed),
                               ptr(workspace),
                               int(nbytes(workspace) if ws_bytes is None else ws_bytes),
                               stream_ptr(stream)), "lbm_batch_run")


def lbm_autotune_save(path):
    check(load().lbm_autotune_save(str(path).encode()), "lbm_autotune_save")


def lbm_autotune_load(path):
    check(load().lbm_autotune_load(str(path).encode()), "lbm_autotune_load")
