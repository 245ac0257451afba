"""Small cases of every kernel family of the fused step, run through the
library that mdf.lib() loads (the release build, or the debug build with
MDF_DEBUG_LIBRARY=1); used by test_gpu_debug_build.py.  `python
tests/debug_cases.py OUT.npz` writes the final states."""
import math
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2306_08216_gb300 import mdf  # noqa: E402
from paper_2306_08216_gb300 import workloads as W  # noqa: E402

LID = dict(walls=(True, True), u_wall=(0, 0, 0, 0.1))


def power_law(re, n_index, u0=0.1):
    K = u0 ** (2 - n_index) / re
    nu = K * u0 ** (n_index - 1)
    return dict(nu=nu, power_law=(K, n_index, nu / 20, nu * 20))


def solo(name, nx, ny, kw, plan, steps=40, init=None, rho0=None):
    s = mdf.Solver(nx, ny, **kw)
    s.set_launch(*plan)
    s.init(*(init if init is not None else W.zeros(nx, ny)))
    if rho0 is not None:
        s.init_rho0(rho0)
    s.step(steps)
    out = {name: s.state()}
    if kw.get("rho0"):
        out[name + "_rho0"] = s.rho0_state()
    return out


def batch(name, probs, kernel, steps=40):
    b = mdf.Batch(probs)
    b.set_launch(kernel)
    b.step(steps)
    return {"%s_%d" % (name, i): b.problem(i).state() for i in range(len(probs))}


def run_cases():
    out = {}
    n = 40
    tg = W.taylor_green(n, 0.02)
    X, Y = np.meshgrid(np.arange(n) / n, np.arange(n) / n)
    rho = 1 + 0.1 * np.sin(2 * math.pi * X) * np.cos(2 * math.pi * Y)
    per = dict(nu=0.01, lx=2 * math.pi, ly=2 * math.pi)
    out.update(solo("fast", n, n, per, (128, 7), init=tg))
    out.update(solo("fast256", n, n, per, (256, 9), init=tg))
    j = np.arange(36)
    y = j / 36 + 0.02 * np.sin(2 * np.pi * j / 36) / (2 * np.pi)
    Xs, Ys = np.meshgrid(W.periodic_nodes(44, 1.0), y)
    forced = dict(nu=0.01, grid="separable", x=W.periodic_nodes(44, 1.0), y=y, lx=1.0, ly=1.0,
                  force=(1e-3 * np.sin(2 * math.pi * Ys), 0 * Ys), force_rate=(1e-4, 0.0),
                  source=0.01 * np.sin(2 * math.pi * Xs))
    out.update(solo("fast_forced", 44, 36, forced, (128, 5)))
    out.update(solo("walls_pl", 33, 33, dict(**LID, **power_law(200, 0.7)), (128, 5)))
    out.update(solo("walls_pl256", 33, 33, dict(**LID, **power_law(200, 1.3)), (256, 6)))
    Xt, Yt = W.trapezoid_grid(33, 33)
    curvi = dict(grid="curvilinear", x=Xt, y=Yt, **LID, **power_law(150, 0.8))
    out.update(solo("curvi_march", 33, 33, curvi, (128, 4)))
    out.update(solo("curvi_tile", 33, 33, curvi, (0, 0)))
    out.update(solo("rho0_fast", n, n, dict(rho0=True, **per), (128, 7), init=tg, rho0=rho))
    out.update(solo("rho0_tile", 33, 33, dict(rho0=True, nu=0.01, **LID), (0, 0)))
    out.update(solo("rho0_march", 33, 33, dict(rho0=True, grid="curvilinear", x=Xt, y=Yt, nu=0.01, **LID), (128, 4)))
    out.update(solo("fp16_fast", n, n, dict(storage="fp16", **per), (256, 9), init=tg))
    out.update(solo("bf16_tile", 33, 33, dict(storage="bf16", **LID, **power_law(200, 0.7)), (0, 0)))
    probs = [dict(nx=s, ny=s, **LID, **power_law(re, ni)) for s, re, ni in ((41, 300, 0.7), (29, 120, 1.2), (50, 500, 1.0))]
    for kernel in ("march", "march_rolled", "tile"):
        out.update(batch("batch_" + kernel, probs, kernel))
    out.update(batch("batch_fp16_rolled", [dict(p, storage="fp16") for p in probs], "march_rolled"))
    mdf.lib()  # the library these ran on
    return out


if __name__ == "__main__":
    states = run_cases()
    np.savez(sys.argv[1], library=os.path.basename(mdf.LIB_PATH), **states)
