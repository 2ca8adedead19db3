"""The C ABI from plain C: tests/c/abi_consumer.c, compiled here with gcc
against include/lbmgnn.h and linked to liblbmgnn.so, calls the library with
no Python in its process.  Its host-only part must agree with the ctypes
binding; its GPU part (a Taylor-Green stack of 2 x 24 x 20 nodes, 7 BGK steps
with totals, then one GNN-LBM step) with the FP64 oracle, at the tolerances
of the other GPU tests (BGK: 3e-6 relative per population after 7 FP32
steps; GNN-LBM: relative L2 of the correction f_gnn - f_bgk <= 3e-2)."""
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2504_14494_gb300 import build
from paper_2504_14494_gb300 import lib as L

HERE = os.path.dirname(os.path.abspath(__file__))
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def consumer(tmp_path_factory):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    lib = build.build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path_factory.mktemp("c") / "abi_consumer")
    cuda_lib = os.path.join(CUDA_HOME, "lib64")
    cmd = [gcc, "-std=c11", "-O2", "-Wall", "-Wextra", "-Werror",
           "-I", os.path.join(build.ROOT, "include"), "-I", os.path.join(CUDA_HOME, "include"),
           os.path.join(HERE, "c", "abi_consumer.c"), "-o", exe,
           "-L", libdir, "-llbmgnn", "-L", cuda_lib, "-lcudart", "-lm",
           f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{cuda_lib}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def _run(exe, *args):
    r = subprocess.run([exe, *args], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_host_calls_from_c_agree_with_the_binding(consumer):
    got = _run(consumer, "host")
    s = L.shape(24, 20, 2)
    assert got["param_count"] == L.gnn_param_count()
    assert got["trainable_count"] == L.gnn_trainable_count()
    assert got["packed_bytes"] == L.gnn_packed_bytes()
    assert got["step_ws"] == L.gnn_step_workspace_bytes(s)
    assert got["channel_ws"] == L.gnn_channel_workspace_bytes(s)
    assert got["host_ws"] == L.lbm_host_workspace_bytes(s)
    assert got["saved_bytes"] == L.gnn_saved_bytes(s)
    theta = L.gnn_params_init_xavier(np.zeros(L.gnn_param_count(), np.float32), 5, 1e-2, 0)
    t64 = theta.astype(np.float64)
    assert got["xavier_sum"] == pytest.approx(float(np.sum(t64)), rel=1e-12, abs=1e-12)
    assert got["xavier_sum_abs"] == pytest.approx(float(np.sum(np.abs(t64))), rel=1e-12)
    assert np.float32(got["xavier_first"]) == theta[0]
    assert np.float32(got["xavier_last"]) == theta[-1]
    assert got["bad_null"] == L.LBM_ERR_ARG and got["bad_variant"] == L.LBM_ERR_ARG
    assert got["status_ok"] == L.status_string(L.LBM_OK)
    assert got["status_tau"] == L.status_string(L.LBM_ERR_TAU)
    assert (got["abi"], got["layout"]) == L.lbm_version()
    assert got["train_ws"] == L.gnn_train_workspace_bytes(s)
    assert got["rollout_ws"] == L.gnn_rollout_workspace_bytes(s, 3)
    assert got["bad_factor"] == L.LBM_ERR_ARG and got["bad_k"] == L.LBM_ERR_ARG


@pytest.mark.gpu
def test_gpu_calls_from_c_match_the_oracle(consumer, tmp_path):
    from oracle import gnn, lbm
    out = tmp_path / "state.bin"
    got = _run(consumer, "gpu", str(out))
    nb, ny, nx = 2, 20, 24
    n = nb * ny * nx
    assert got["nodes"] == n
    assert got["alias"] == L.LBM_ERR_ALIAS
    raw = out.read_bytes()
    fb = 9 * n * 4
    bgk = np.frombuffer(raw[:fb], np.float32).reshape(9, nb, ny, nx).astype(np.float64)
    tot = np.frombuffer(raw[fb:fb + 40], np.float64)
    gstate = np.frombuffer(raw[fb + 40:2 * fb + 40], np.float32).reshape(9, nb, ny, nx)
    gstate = gstate.astype(np.float64)
    cstate = np.frombuffer(raw[2 * fb + 40:], np.float32).reshape(9, nb, ny, nx).astype(np.float64)
    f0 = lbm.tgv_init(nx, ny, 1.0, 0.05, 2 * np.pi / nx, 2 * np.pi / ny)
    ref = lbm.bgk_run(f0, 0.7, 7)
    for b in range(nb):
        assert np.allclose(bgk[:, b], ref, rtol=3e-6, atol=0)
    assert tot[0] == pytest.approx(float(np.sum(bgk)), rel=1e-12)
    assert tot[4] == 0.0
    theta = L.gnn_params_init_xavier(np.zeros(L.gnn_param_count(), np.float32), 5, 1e-2, 0)
    for b in range(nb):
        want = gnn.gnn_step(bgk[:, b], theta.astype(np.float64), 0.7)
        plain = lbm.bgk_step(bgk[:, b], 0.7)
        d, w = gstate[:, b] - plain, want - plain
        assert float(np.sqrt(np.sum((d - w) ** 2) / np.sum(w ** 2))) <= 3e-2
    from oracle import channel
    for b in range(nb):  # the channel's GNN-LBM step of the same state
        want = channel.gnn_channel_step(bgk[:, b], theta.astype(np.float64), 0.7, 1e-4)
        plain = channel.channel_step(bgk[:, b], 0.7, 1e-4)
        d, w = cstate[:, b] - plain, want - plain
        assert float(np.sqrt(np.sum((d - w) ** 2) / np.sum(w ** 2))) <= 3e-2
