"""Microbenchmarks that fix the peaks behind the roofline fractions of the
tensor-core and packed-FP16 kernels (run on the GPU):

    python -m paper_2504_14494_gb300.microbench          # builds with nvcc, runs, prints JSON

mma_rate.cu: cycles per tcgen05.mma (M = 128, K = 16, BF16) for N = 16..256
with one and two CTAs per SM; fp16_rate.cu: warp instructions per clock per
SM of HFMA2, tanh.approx.f16x2 and the edge-message sequence of the
message-passing round (7 packed-FP16 operations and one tanh per pair of
edge-feature GELUs).
"""
import json
import os
import subprocess
import sys

from . import build

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "microbench")


def _build(name):
    out = os.path.join(build.OBJDIR, name)
    os.makedirs(build.OBJDIR, exist_ok=True)
    src = os.path.join(HERE, name + ".cu")
    cmd = [build._nvcc(), *build.ARCH, "-O3", "-std=c++17", "-I", build.CSRC, src, "-o", out]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return out


def run():
    res = {}
    exe = _build("fp16_rate")
    res["fp16"] = json.loads(subprocess.run([exe], check=True, capture_output=True,
                                            text=True).stdout.strip().splitlines()[-1])
    exe = _build("mma_rate")
    res["tcgen05_mma"] = subprocess.run([exe], check=True, capture_output=True,
                                        text=True).stdout.strip().splitlines()
    return res


if __name__ == "__main__":
    json.dump(run(), sys.stdout)
    print()
