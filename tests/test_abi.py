"""The C ABI library builds, loads and exports every entry point declared in
include/*.h; host-side argument checks return their codes without touching a
GPU (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2504_14494_gb300 import lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names += re.findall(r"LBM_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lbmlib):
    names = _declared()
    assert "lbm_step_bgk" in names and len(names) >= 5
    so = ctypes.CDLL(L.LIB_PATH)
    for n in names:
        assert hasattr(so, n), n


def test_binding_covers_every_declared_symbol(lbmlib):
    assert set(_declared()) <= set(L.exported_symbols())


def test_status_strings(lbmlib):
    for code in range(0, -11, -1):
        s = L.status_string(code)
        assert s and s != "unknown status"
    assert L.status_string(-99) == "unknown status"


def test_host_argument_checks(lbmlib):
    so = L.load()
    s = L.shape(8, 8)
    # NULL buffers
    assert so.lbm_step_bgk(None, 1 << 20, None, s, 0.8, None, 1, None, None) == -1
    # bad sizes and plane stride
    assert so.lbm_step_bgk(1 << 20, 1 << 24, None, L.shape(0, 8), 0.8, None, 1, None, None) == -3
    assert so.lbm_step_bgk(1 << 20, 1 << 24, None, L.shape(8, 8, 1, 10), 0.8, None, 1, None, None) == -3
    # in == out, overlapping tmp
    assert so.lbm_step_bgk(1 << 20, 1 << 20, None, s, 0.8, None, 1, None, None) == -2
    assert so.lbm_step_bgk(1 << 20, 1 << 24, (1 << 20) + 64, s, 0.8, None, 2, None, None) == -2
    # missing tmp for nsteps > 1, negative steps
    assert so.lbm_step_bgk(1 << 20, 1 << 24, None, s, 0.8, None, 2, None, None) == -1
    assert so.lbm_step_bgk(1 << 20, 1 << 24, None, s, 0.8, None, -1, None, None) == -1
    # tau <= 1/2 or NaN
    assert so.lbm_step_bgk(1 << 20, 1 << 24, None, s, 0.5, None, 1, None, None) == -4
    assert so.lbm_step_bgk(1 << 20, 1 << 24, None, s, float("nan"), None, 1, None, None) == -4
    assert so.lbm_init_tgv(None, s, 1.0, 0.01, 0.1, 0.1, 0, None) == -1
    assert so.lbm_init_tgv(1 << 20, s, -1.0, 0.01, 0.1, 0.1, 0, None) == -1
    assert so.lbm_moments(None, s, None, None, None, None, None) == -1
    # GNN step of the channel: workspace size, force, tau, aliasing
    need = L.gnn_channel_workspace_bytes(s)
    assert need == ((9 * 64 * 4 + 255) // 256) * 256 + 808 * 64
    assert L.gnn_channel_workspace_bytes(L.shape(0, 8)) == 0
    a, b, pk, ws = 1 << 20, 1 << 24, 1 << 28, 1 << 32
    assert so.lbm_step_gnn_channel(a, b, s, 0.8, None, 1e-3, pk, None, ws, need - 1, None) == -10
    assert so.lbm_step_gnn_channel(a, b, s, 0.8, None, 1e-3, pk, None, ws + 16, need, None) == -10
    assert so.lbm_step_gnn_channel(a, b, s, 0.8, None, float("nan"), pk, None, ws, need,
                                   None) == -1
    assert so.lbm_step_gnn_channel(a, b, s, 0.5, None, 1e-3, pk, None, ws, need, None) == -4
    assert so.lbm_step_gnn_channel(a, a, s, 0.8, None, 1e-3, pk, None, ws, need, None) == -2
    assert so.lbm_step_gnn_channel(a, b, s, 0.8, None, 1e-3, pk, None, a + 256, need, None) == -2
    # forced restriction of a refined channel: odd factor, sizes, force, tau, aliasing
    fine, coarse = L.shape(24, 24), L.shape(8, 8)
    assert so.lbm_restrict_channel(a, L.shape(16, 16), b, coarse, 2, 0.8, None, 0.7, None, 1e-4,
                                   None, None) == -1
    assert so.lbm_restrict_channel(a, L.shape(24, 21), b, coarse, 3, 0.8, None, 0.7, None, 1e-4,
                                   None, None) == -3
    assert so.lbm_restrict_channel(a, fine, b, coarse, 3, 0.8, None, 0.7, None, float("inf"),
                                   None, None) == -1
    assert so.lbm_restrict_channel(a, fine, b, coarse, 3, 0.8, None, 0.5, None, 1e-4, None,
                                   None) == -4
    assert so.lbm_restrict_channel(a, fine, a + 256, coarse, 3, 0.8, None, 0.7, None, 1e-4, None,
                                   None) == -2
    assert so.lbm_restrict_channel(None, fine, b, coarse, 3, 0.8, None, 0.7, None, 1e-4, None,
                                   None) == -1
    # channel training step: force, tau, workspace
    tw = L.gnn_train_workspace_bytes(s)
    prm, m_, v_, loss = 1 << 33, 1 << 34, 1 << 35, 1 << 36
    args = lambda tau, fx, wsb: (a, b, s, tau, None, fx, None, None, prm, pk, m_, v_, 1, 1e-3,
                                 1e-2, loss, None, ws, wsb, None)
    assert so.gnn_train_step_channel(*args(0.8, float("nan"), tw)) == -1
    assert so.gnn_train_step_channel(*args(0.5, 1e-4, tw)) == -4
    assert so.gnn_train_step_channel(*args(0.8, 1e-4, tw - 1)) == -10
    # K-step rollout training step: K range, workspace
    assert L.gnn_rollout_workspace_bytes(s, 0) == 0 and L.gnn_rollout_workspace_bytes(s, 65) == 0
    rw = L.gnn_rollout_workspace_bytes(s, 2)
    assert rw > 2 * 64 * 1152
    rargs = lambda k, wsb: (a, b, k, s, 0.8, None, prm, pk, m_, v_, 1, 1e-3, 1e-2, loss, None, ws,
                            wsb, None)
    assert so.gnn_train_step_rollout(*rargs(0, rw)) == -1
    assert so.gnn_train_step_rollout(*rargs(65, rw)) == -1
    assert so.gnn_train_step_rollout(*rargs(2, rw - 1)) == -10


def test_binding_raises_on_error(lbmlib):
    with pytest.raises(L.LbmError) as ei:
        L.lbm_step_bgk(None, None, None, L.shape(4, 4), 0.8, stream=0)
    assert ei.value.code == -1


def test_versions(lbmlib):
    """lbm_version: the ABI and packed-layout versions the header declares."""
    L = lbmlib
    header = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                               "include", "lbmgnn.h")).read()
    abi = int(re.search(r"#define LBM_ABI_VERSION (\d+)", header).group(1))
    layout = int(re.search(r"#define LBM_PACKED_LAYOUT_VERSION (\d+)", header).group(1))
    assert L.lbm_version() == (abi, layout)
    assert L.load().lbm_version(None, None) == L.LBM_OK
