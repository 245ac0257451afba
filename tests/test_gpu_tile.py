"""GPU parity of the tile kernel (one block per 16 x 16 tile, three phases,
recomputed halo) against the FP64 oracle, for every grid kind, wall layout
and fluid model, on grid sizes that leave ragged tiles; and its agreement
with the marches.  Tolerance: the FP32 parity bar, 1e-5 of the reference
velocity."""
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


def maxabs(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max())


def run_tile(nx, ny, steps, init, **kw):
    g, o = mdf.Solver(nx, ny, **kw), Oracle(nx, ny, **kw)
    g.set_launch(0)
    assert g.launch_info()["kernel"] == "tile"
    for s in (g, o):
        s.init(*init)
    g.step(steps)
    o.step(steps)
    return g, o


@pytest.mark.parametrize("nx,ny", [(5, 5), (12, 9), (33, 33), (45, 31), (70, 17)])
@pytest.mark.parametrize("walls", [(False, False), (True, True), (False, True), (True, False)])
def test_ragged_grids_and_wall_layouts(nx, ny, walls):
    U0 = 0.02
    kw = dict(nu=0.02, walls=walls, u_wall=(0.01, -0.01, 0.0, U0), v_wall=(0.0, 0.0, 0.005, 0.0))
    if not walls[0]:
        kw["lx"] = 1.0
    if not walls[1]:
        kw["ly"] = ny / nx
    g, o = run_tile(nx, ny, 120, W.random_fields(nx, ny, U0, 3), **kw)
    assert maxabs(g.state(), o.state()) <= 1e-5 * U0


def test_taylor_green_64_after_1000_steps():
    n, U0 = 64, 0.01
    g, o = run_tile(n, n, 1000, W.taylor_green(n, U0), nu=0.01, lx=2 * math.pi, ly=2 * math.pi)
    assert maxabs(g.state(), o.state()) <= 1e-5 * U0


def test_lid_driven_cavity_after_1000_steps():
    n, U0 = 65, 0.1
    g, o = run_tile(n, n, 1000, W.zeros(n, n), nu=0.01, walls=(True, True), u_wall=(0, 0, 0, U0))
    assert maxabs(g.state(), o.state()) <= 1e-5 * U0


@pytest.mark.parametrize("n_index", [0.6, 1.4])
def test_power_law_cavity(n_index):
    n, U0 = 49, 0.1
    K = 0.01 * U0 ** (1 - n_index)
    kw = dict(nu=0.01, walls=(True, True), u_wall=(0, 0, 0, U0), power_law=(K, n_index, 5e-4, 0.2))
    g, o = run_tile(n, n, 400, W.zeros(n, n), **kw)
    assert maxabs(g.state(), o.state()) <= 1e-5 * U0


def test_tanh_stretched_cavity():
    n, U0 = 41, 0.1
    x = 0.5 * (1 + np.tanh(1.5 * (2 * np.arange(n) / (n - 1) - 1)) / np.tanh(1.5))
    kw = dict(nu=0.01, grid="separable", x=x, y=x, walls=(True, True), u_wall=(0, 0, 0, U0))
    g, o = run_tile(n, n, 400, W.zeros(n, n), **kw)
    assert maxabs(g.state(), o.state()) <= 1e-5 * U0


@pytest.mark.parametrize("power_law", [None, (0.002, 0.7, 1e-4, 0.05)])
def test_trapezoid_cavity_curvilinear(power_law):
    n, U0 = 37, 0.1
    X, Y = W.trapezoid_grid(n, n)
    kw = dict(nu=0.01, grid="curvilinear", x=X, y=Y, walls=(True, True), u_wall=(0, 0, 0, U0))
    if power_law:
        kw["power_law"] = power_law
    g, o = run_tile(n, n, 300, W.zeros(n, n), **kw)
    assert maxabs(g.state(), o.state()) <= 1e-5 * U0


def test_periodic_separable_with_force_rate_and_source_fields():
    nx, ny, nu = 40, 24, 0.02
    j = np.arange(ny)
    y = j / ny + 0.02 * np.sin(2 * np.pi * j / ny) / (2 * np.pi)
    Xg, Yg = np.meshgrid(np.arange(nx) / nx, y)
    F = (1e-4 * np.sin(2 * np.pi * Yg), 5e-5 * np.cos(2 * np.pi * Xg))
    dF = (-1e-5 * np.cos(2 * np.pi * Xg), 2e-5 * np.sin(2 * np.pi * Yg))
    R = 0.01 * np.sin(2 * np.pi * Xg) * np.cos(2 * np.pi * Yg)
    kw = dict(nu=nu, grid="separable", x=W.periodic_nodes(nx, 1.0), y=y, lx=1.0, ly=1.0, force=F, force_rate=dF,
              source=R)
    g, o = run_tile(nx, ny, 300, W.zeros(nx, ny), **kw)
    ref = 1e-4 / (nu * (2 * np.pi) ** 2)
    assert maxabs(g.state(), o.state()) <= 1e-5 * max(ref, 0.01)


def test_tile_and_march_agree():
    """The two kernel families on the same power-law cavity: both within
    the parity bar of the oracle, and within a few FP32 roundings of each
    other."""
    n, U0 = 90, 0.1
    kw = dict(nu=0.004, walls=(True, True), u_wall=(0, 0, 0, U0), power_law=(0.004, 0.8, 2e-4, 0.08))
    a, b = mdf.Solver(n, n, **kw), mdf.Solver(n, n, **kw)
    a.set_launch(0)
    b.set_launch(128, 6)
    for s in (a, b):
        s.init(*W.zeros(n, n))
        s.step(500)
    assert maxabs(a.state(), b.state()) <= 1e-6 * U0


def test_graph_replay_and_checkpoint_on_the_tile_kernel(tmp_path):
    n = 33
    kw = dict(nu=0.01, walls=(True, True), u_wall=(0, 0, 0, 0.1))
    a, b = mdf.Solver(n, n, **kw), mdf.Solver(n, n, **kw)
    for s in (a, b):
        s.set_launch(0)
        s.init(*W.zeros(n, n))
    a.step(50)
    for _ in range(50):
        b.step(1)
    np.testing.assert_array_equal(a.state(), b.state())
    a.save(tmp_path / "t.ckpt")
    a.step(20)
    c = mdf.Solver(n, n, **kw)
    c.set_launch(0)
    c.load(tmp_path / "t.ckpt")
    c.step(20)
    np.testing.assert_array_equal(a.state(), c.state())


def test_autotuner_prefers_the_tile_kernel_on_a_small_cavity():
    """257^2 Re 1000 cavity: print the chosen plan and its step time next
    to the best march (the choice itself is a timing, not asserted)."""
    n = 257
    kw = dict(nu=1e-4, walls=(True, True), u_wall=(0, 0, 0, 0.1))
    s = mdf.Solver(n, n, **kw)
    info = s.launch_info()
    times = {}
    for plan in ("auto", "tile", "march"):
        if plan == "tile":
            s.set_launch(0)
        elif plan == "march":
            s.set_launch(128, 2)
        s.init(*W.zeros(n, n))
        s.step(64)
        s.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.step(640)
        e1.record()
        e1.synchronize()
        times[plan] = e0.elapsed_time(e1) / 640 * 1e3
    print("257^2 cavity: autotuned %s, us per step %s" % (info["kernel"], times))
    assert info["kernel"] in ("tile", "march")
