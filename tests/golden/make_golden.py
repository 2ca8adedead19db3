"""Writes the stored expected values under tests/golden/ from the FP64 oracle.

Run from the repository root:  python tests/golden/make_golden.py
It calls only the oracle package; no value comes from the CUDA library.
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import lbm  # noqa: E402


def tgv64():
    """64^2 periodic TGV, tau=0.8, u0=0.01, k=2 pi/64, rho0=1, 1000 steps."""
    n, u0, tau, steps = 64, 0.01, 0.8, 1000
    k = 2 * np.pi / n
    f = lbm.tgv_init(n, n, 1.0, u0, k, k)
    t0 = lbm.totals(f)
    f = lbm.bgk_run(f, tau, steps)
    rho, ux, uy = lbm.moments(f)
    err = lbm.velocity_l2_error(ux, uy, *lbm.tgv_analytic_velocity(n, n, u0, k, k, tau, steps))
    return {"n": n, "u0": u0, "tau": tau, "steps": steps, "rho0": 1.0,
            "l2_error": err, "totals0": t0.tolist(), "totals": lbm.totals(f).tolist(),
            "source": "oracle.lbm, FP64; Sec. 3.2 TGV workload"}


if __name__ == "__main__":
    with open(os.path.join(HERE, "tgv64_bgk.json"), "w") as fh:
        json.dump(tgv64(), fh, indent=1)
    print("wrote", os.path.join(HERE, "tgv64_bgk.json"))
