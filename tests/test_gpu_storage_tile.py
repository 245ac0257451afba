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


def batch_problems(mode):
    probs = []
    for side, re, ni in [(65, 400, 0.6), (33, 100, 1.0), (47, 250, 1.4)]:
        K = 0.1 ** (2 - ni) / re
        probs.append(dict(nx=side, ny=side, nu=K * 0.1 ** (ni - 1), walls=(True, True), u_wall=(0, 0, 0, 0.1),
                          power_law=(K, ni, K * 0.1 ** (ni - 1) / 20, K * 0.1 ** (ni - 1) * 20), storage=mode))
    return probs


@pytest.mark.parametrize("mode", MODES)
def test_batch_equals_solo_runs_bitwise(mode):
    """In tile mode a 16-bit batch computes what the same problems compute
    alone (single 16-bit problems with walls step on the tile kernel)."""
    probs = batch_problems(mode)
    batch = mdf.Batch(probs)
    assert batch.info()["kernel"] in ("tile", "march_rolled")
    batch.set_launch("tile")
    batch.step(40)
    for i, kw in enumerate(probs):
        kw = dict(kw)
        nx, ny = kw.pop("nx"), kw.pop("ny")
        solo = mdf.Solver(nx, ny, **kw)
        solo.init(*W.zeros(nx, ny))
        solo.step(40)
        np.testing.assert_array_equal(batch.problem(i).state(), solo.state())


@pytest.mark.parametrize("mode", MODES)
def test_batch_rolled_march_against_oracle(mode):
    """The rolled wall/power-law march with 16-bit storage (batches on
    uniform grids): every problem within the N-step bound of the oracle,
    N 15 u_r max|n| plus the 5e-7 U0 of the FP32 path; the tile-mode batch
    within the same bound."""
    probs = batch_problems(mode)
    steps, U0 = 120, 0.1
    states = {}
    for kind in ("march_rolled", "tile"):
        b = mdf.Batch(probs)
        b.set_launch(kind)
        assert b.info()["kernel"] == kind
        b.step(steps)
        states[kind] = [b.problem(i).state() for i in range(len(probs))]
    for i, kw in enumerate(probs):
        kw = dict(kw)
        nx, ny = kw.pop("nx"), kw.pop("ny")
        kw.pop("storage")
        o = Oracle(nx, ny, **kw)
        o.init(*W.zeros(nx, ny))
        o.step(steps)
        nmax = noneq_max(o)
        bound = 5e-7 * U0 + steps * 15 * UNIT_ROUNDOFF[mode] * nmax
        for kind, st in states.items():
            err = maxabs(st[i], o.state())
            assert err <= bound, (kind, i, err, bound)


@pytest.mark.parametrize("mode", MODES)
def test_batch_rolled_march_poisoned_equals_clean(mode):
    """NaN in every storage element no valid result may read (row padding,
    ghost columns beside x walls) changes nothing in the 16-bit rolled march."""
    probs = batch_problems(mode)
    out = []
    for poison in (False, True):
        b = mdf.Batch(probs)
        b.set_launch("march_rolled")
        if poison:
            for i in range(len(probs)):
                b.problem(i).debug_poison()
        b.step(40)
        b.step(3)
        out.append([b.problem(i).state() for i in range(len(probs))])
    for a, c in zip(*out):
        assert np.isfinite(c).all()
        np.testing.assert_array_equal(a, c)


def test_16bit_batch_rejects_the_unrolled_march():
    b = mdf.Batch(batch_problems("fp16"))
    with pytest.raises(mdf.MdfError) as e:
        b.set_launch("march")
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
