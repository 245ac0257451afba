"""Full-size, long-run parity of the benchmark workloads against the FP64
oracle, in the launch configurations the benchmark times (the autotuned
single-problem plans; the batch as created), after 1000 steps from rest:

  * the Re = 1000 lid-driven cavity on 257 x 257 nodes, uniform and
    tanh-stretched (beta = 1.5) grids;
  * power-law lid-driven cavities on the 513 x 513 body-fitted trapezoid
    (n = 0.5 at Re = 1000, n = 1.5 at Re = 100);
  * the seeded 512-cavity sweep stepped as one batch, the first cavity of
    every side (65, 129, 257, 513) checked.

The bar is the FP32 parity bar, max |GPU - oracle| <= 1e-5 times the lid
speed over every distribution of every node.  The oracle runs the full grid
(its OpenMP threads), about 10 s per 1000 steps of a 257^2 Newtonian cavity
and 1-2 min per 1000 steps of a 513^2 power-law one."""
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
U0 = 0.1
STEPS = 1000


def power_law_cavity(n_index, re, u0=U0):
    """K from Re = u0^(2-n) L^n / K with L = 1; nu clamped to [nu_ref/20, 20 nu_ref]."""
    K = u0 ** (2.0 - n_index) / re
    nu_ref = K * u0 ** (n_index - 1.0)
    return dict(nu=nu_ref, walls=(True, True), u_wall=(0, 0, 0, u0),
                power_law=(K, float(n_index), nu_ref / 20, nu_ref * 20))


def max_state_error(g_state, o):
    return float(np.abs(g_state.astype(np.float64) - o.state()).max())


@pytest.mark.parametrize("grid", ["uniform", "tanh"])
def test_cavity_257_re1000_after_1000_steps(grid):
    """The time-to-residual workload (Re = 1000, u0 = 0.1, nu = 1e-4), the
    tanh grid with its ~3.3 x shorter time step."""
    n = 257
    kw = dict(nu=U0 / 1000.0, walls=(True, True), u_wall=(0, 0, 0, U0))
    if grid == "tanh":
        xs = W.tanh_nodes(n, 1.5)
        kw.update(grid="separable", x=xs, y=xs)
    g, o = mdf.Solver(n, n, **kw), Oracle(n, n, **kw)
    assert abs(g.dt - o.dt) <= 1e-12 * o.dt
    for s in (g, o):
        s.init(*W.zeros(n, n))
    g.step(STEPS)
    o.step(STEPS)
    err = max_state_error(g.state(), o)
    assert err <= 1e-5 * U0, err
    fg, fo = g.fields(["u", "v"]), o.fields()
    assert float(np.abs(fg["u"] - fo["u"]).max()) <= 1e-5 * U0


@pytest.mark.parametrize("n_index,re", [(0.5, 1000.0), (1.5, 100.0)])
def test_trapezoid_513_power_law_after_1000_steps(n_index, re):
    n = 513
    X, Y = W.trapezoid_grid(n, n)
    kw = dict(grid="curvilinear", x=X, y=Y, **power_law_cavity(n_index, re))
    g, o = mdf.Solver(n, n, **kw), Oracle(n, n, **kw)
    for s in (g, o):
        s.init(*W.zeros(n, n))
    g.step(STEPS)
    o.step(STEPS)
    err = max_state_error(g.state(), o)
    assert err <= 1e-5 * U0, err
    fg, fo = g.fields(["nu"]), o.fields()
    np.testing.assert_allclose(fg["nu"], fo["nu"], rtol=2e-3)


def test_512_cavity_batch_after_1000_steps():
    """The seeded sweep (sides 65-513, Re 100-5000, n 0.5-1.5) stepped as one
    batch for 1000 steps; the first problem of every side against the oracle."""
    re, nn, sides = W.cavity_batch_draws(512, 2306)
    probs = [dict(nx=int(sd), ny=int(sd), **power_law_cavity(float(b), float(a))) for a, b, sd in zip(re, nn, sides)]
    batch = mdf.Batch(probs)
    batch.step(STEPS)
    info = batch.info()
    assert info["problems"] == 512 and info["steps"] == STEPS
    checked = 0
    for side in (65, 129, 257, 513):
        i = int(np.nonzero(sides == side)[0][0])
        kw = dict(probs[i])
        nx, ny = kw.pop("nx"), kw.pop("ny")
        o = Oracle(nx, ny, **kw)
        o.init(*W.zeros(nx, ny))
        o.step(STEPS)
        err = max_state_error(batch.problem(i).state(), o)
        assert err <= 1e-5 * U0, (side, float(re[i]), float(nn[i]), err)
        checked += 1
    assert checked == 4
