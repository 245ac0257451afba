"""16-bit deviation storage (FP32 u, v, P plus FP16 / BF16 non-equilibrium
parts, FP32 arithmetic) on the problems the tile kernel serves: walls, power
law, curvilinear grids, and batches of cavities.  Bounds as for the periodic
fast path: one step from an oracle state to 5e-7 U0 + 16 u_r max|n| (the
input rounding plus its image through one step); N steps to the per-step
bound summed, N 15 u_r max|n|; and, for a lid-driven cavity, the distance
from the FP32 run."""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2306_08216_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2306_08216_gb300 import build as B  # noqa: E402
from paper_2306_08216_gb300 import mdf  # noqa: E402

B.build()

UNIT_ROUNDOFF = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}
MODES = ["fp16", "bf16"]


def feq(u, v, P, c=1.0):
    """Linear equilibrium of Eq. 2.2.5 on D2Q5, layout [alpha][j][ny][nx]."""
    out = np.zeros((2, 5) + u.shape)
    for a, (ub, fx, fy) in enumerate([(u, u * u + P, u * v), (v, u * v, v * v + P)]):
        out[a, 0] = ub / 5
        out[a, 1] = ub / 5 + fx / (2 * c)
        out[a, 3] = ub / 5 - fx / (2 * c)
        out[a, 2] = ub / 5 + fy / (2 * c)
        out[a, 4] = ub / 5 - fy / (2 * c)
    return out


def noneq_max(o):
    s, f = o.state(), o.fields()
    return float(np.abs(s - feq(f["u"], f["v"], f["P"])).max())


def maxabs(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max())


def cavity_kw(kind):
    U0 = 0.1
    kw = dict(nu=0.01, walls=(True, True), u_wall=(0, 0, 0, U0))
    if kind == "power_law":
        kw["power_law"] = (0.01 * U0 ** 0.4, 0.6, 5e-4, 0.2)
    elif kind == "curvilinear":
        X, Y = W.trapezoid_grid(41, 41)
        kw.update(grid="curvilinear", x=X, y=Y)
    return kw, U0


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("kind", ["newtonian", "power_law", "curvilinear"])
def test_one_step_from_an_oracle_state(mode, kind):
    n = 41
    kw, U0 = cavity_kw(kind)
    o = Oracle(n, n, **kw)
    o.init(*W.zeros(n, n))
    o.step(200)
    s0, nmax = o.state(), noneq_max(o)
    g = mdf.Solver(n, n, storage=mode, **kw)
    assert g.launch_info()["kernel"] == "tile"
    g.set_state(s0.astype(np.float32))
    g.step(1)
    o.step(1)
    err = maxabs(g.state(), o.state())
    assert err <= 5e-7 * U0 + 16 * UNIT_ROUNDOFF[mode] * nmax, (err, nmax)


@pytest.mark.parametrize("mode", MODES)
def test_cavity_400_steps_against_oracle_and_fp32(mode):
    n = 41
    kw, U0 = cavity_kw("power_law")
    o = Oracle(n, n, **kw)
    g16, g32 = mdf.Solver(n, n, storage=mode, **kw), mdf.Solver(n, n, **kw)
    for s in (o, g16, g32):
        s.init(*W.zeros(n, n))
    steps, nmax = 400, 0.0
    for _ in range(4):
        for s in (o, g16, g32):
            s.step(steps // 4)
        nmax = max(nmax, noneq_max(o))
    err = maxabs(g16.state(), o.state())
    assert err <= 5e-7 * U0 + steps * 15 * UNIT_ROUNDOFF[mode] * nmax, (err, nmax)
    du = maxabs(g16.fields(["u"])["u"], g32.fields(["u"])["u"])
    print("%s cavity: max |u16 - u32| = %.2e U0, max|n| = %.2e" % (mode, du / U0, nmax))
    assert du <= (2e-3 if mode == "fp16" else 2e-2) * U0


@pytest.mark.parametrize("mode", MODES)
def test_batch_equals_solo_runs_bitwise(mode):
    probs = []
    for side, re, ni in [(65, 400, 0.6), (33, 100, 1.0), (47, 250, 1.4)]:
        K = 0.1 ** (2 - ni) / re
        probs.append(dict(nx=side, ny=side, nu=K * 0.1 ** (ni - 1), walls=(True, True), u_wall=(0, 0, 0, 0.1),
                          power_law=(K, ni, K * 0.1 ** (ni - 1) / 20, K * 0.1 ** (ni - 1) * 20), storage=mode))
    batch = mdf.Batch(probs)
    assert batch.info()["kernel"] == "tile"
    batch.step(40)
    for i, kw in enumerate(probs):
        kw = dict(kw)
        nx, ny = kw.pop("nx"), kw.pop("ny")
        solo = mdf.Solver(nx, ny, **kw)
        solo.init(*W.zeros(nx, ny))
        solo.step(40)
        np.testing.assert_array_equal(batch.problem(i).state(), solo.state())
    with pytest.raises(mdf.MdfError) as e:
        batch.set_launch("march")
    assert e.value.status == mdf.MDF_E_INVALID


@pytest.mark.parametrize("mode", MODES)
def test_checkpoint_resume_with_walls_is_bitwise(tmp_path, mode):
    n = 37
    kw, _ = cavity_kw("newtonian")
    a = mdf.Solver(n, n, storage=mode, **kw)
    a.init(*W.zeros(n, n))
    a.step(30)
    a.save(tmp_path / "w.ckpt")
    a.step(20)
    b = mdf.Solver(n, n, storage=mode, **kw)
    b.load(tmp_path / "w.ckpt")
    b.step(20)
    np.testing.assert_array_equal(a.state(), b.state())
    assert b.bytes_per_node() == 56.0
