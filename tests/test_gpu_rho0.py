"""GPU parity of the alpha = 0 distribution of Eq. 2.1.2 (ubar_0 = rho_0,
E_0 = 0, source w_j R), evolved beside alpha = 1, 2 on request, against the
FP64 oracle.

Tolerances: rho_0 and its distributions to 1e-5 of max |rho_0| (the FP32
parity bar relative to the field's scale, as the velocity distributions are
held to 1e-5 of the reference velocity); the alpha = 1, 2 state to the
usual bar, 1e-5 of the reference velocity.  Remark 1 (no feedback) is
checked bitwise where the same kernel runs with and without the lane."""
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


def check(g, o, uref):
    r0 = o.rho0()
    bar = 1e-5 * float(np.abs(r0).max())
    assert maxabs(g.rho0_state(), o.rho0_state()) <= bar, maxabs(g.rho0_state(), o.rho0_state())
    assert maxabs(g.rho0(), r0) <= bar
    assert maxabs(g.state(), o.state()) <= 1e-5 * uref


def both(nx, ny, **kw):
    return mdf.Solver(nx, ny, rho0=True, **kw), Oracle(nx, ny, rho0=True, **kw)


@pytest.mark.parametrize("c", [1.0, 2.0])
def test_fourier_mode_in_uniform_flow(c):
    """A Fourier mode of rho_0 carried and diffused by a uniform flow
    (periodic uniform grid), 2 time units as in the oracle's closed-form pin."""
    n, ny, U, e = 64, 8, 0.05, 0.01
    X = np.tile(np.arange(n) / n, (ny, 1))
    g, o = both(n, ny, nu=0.01, lx=1.0, ly=ny / n, c=c)
    z = np.zeros((ny, n))
    for s in (g, o):
        s.init(np.full((ny, n), U), z, z)
        s.init_rho0(1 + e * np.sin(2 * math.pi * X))
    steps = int(round(2.0 / o.dt))
    g.step(steps)
    o.step(steps)
    check(g, o, U)
    t = steps * o.dt
    exact = 1 + e * np.sin(2 * math.pi * (X - U * t)) * math.exp(-0.01 * (2 * math.pi) ** 2 * t)
    assert np.abs(g.rho0() - exact).max() <= 1e-2 * e * (1.0 if c == 1.0 else 0.3)


def test_taylor_green_with_a_scalar_blob():
    n, U0 = 48, 0.02
    kw = dict(nu=0.01, lx=2 * math.pi, ly=2 * math.pi)
    g, o = both(n, n, **kw)
    X, Y = np.meshgrid(np.arange(n) / n, np.arange(n) / n)
    rho = 1 + 0.2 * np.exp(-((X - 0.4) ** 2 + (Y - 0.6) ** 2) / 0.02)
    for s in (g, o):
        s.init(*W.taylor_green(n, U0))
        s.init_rho0(rho)
    g.step(300)
    o.step(300)
    check(g, o, U0)


def test_rest_with_a_uniform_source():
    """At rest with R = 0.02: rho_0 = 1 + R t (the oracle's exact pin)."""
    g, o = both(16, 16, nu=0.01, source=0.02)
    for s in (g, o):
        s.init(*W.zeros(16, 16))
    g.step(100)
    o.step(100)
    check(g, o, 0.02)
    np.testing.assert_allclose(g.rho0(), 1.0 + 0.02 * 100 * o.dt, rtol=2e-6)


@pytest.mark.parametrize("grid", ["uniform", "curvilinear"])
def test_lid_driven_cavity(grid):
    n, U0 = 33, 0.1
    kw = dict(nu=0.01, walls=(True, True), u_wall=(0, 0, 0, U0))
    if grid == "curvilinear":
        X, Y = W.trapezoid_grid(n, n)
        kw.update(grid="curvilinear", x=X, y=Y)
    g, o = both(n, n, **kw)
    Xn, Yn = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n))
    for s in (g, o):
        s.init(*W.zeros(n, n))
        s.init_rho0(1 + 0.1 * np.sin(math.pi * Xn) * np.sin(math.pi * Yn))
    g.step(400)
    o.step(400)
    check(g, o, U0)


def test_power_law_cavity():
    n, U0 = 33, 0.1
    kw = dict(nu=0.01, walls=(True, True), u_wall=(0, 0, 0, U0), power_law=(0.01 * 0.1 ** 0.4, 0.6, 5e-4, 0.2))
    g, o = both(n, n, **kw)
    for s in (g, o):
        s.init(*W.zeros(n, n))
    g.step(300)
    o.step(300)
    check(g, o, U0)


def test_channel_with_source_field_on_a_separable_grid():
    """Walls in y only (x periodic), a stretched separable grid, a body
    force and a source field: every term of the lane at once."""
    nx, ny, U0 = 40, 24, 0.05
    j = np.arange(ny)
    y = 0.5 - 0.5 * np.cos(math.pi * j / (ny - 1))
    X, Y = np.meshgrid(np.arange(nx) / nx, y)
    R = 0.01 * np.sin(2 * math.pi * X) * np.sin(math.pi * Y)
    kw = dict(nu=0.02, grid="separable", x=W.periodic_nodes(nx, 1.0), y=y, lx=1.0, walls=(False, True),
              force=(1e-3, 0.0), source=R)
    g, o = both(nx, ny, **kw)
    for s in (g, o):
        s.init(*W.zeros(nx, ny))
    g.step(300)
    o.step(300)
    check(g, o, U0)


@pytest.mark.parametrize("plan", [(128, 3), (0, 0)])
def test_no_feedback_into_alpha_1_2_bitwise(plan):
    """Remark 1: with the same kernel with and without the lane (the tile
    kernel on any grid; the shared-ring march on a curvilinear grid) the
    alpha = 1, 2 state is identical to the bit; a uniform cavity with the
    march (other kernels without the lane) agrees to the parity bar."""
    n, U0 = 33, 0.1
    X, Y = W.trapezoid_grid(n, n)
    base = dict(nu=0.01, walls=(True, True), u_wall=(0, 0, 0, U0))
    for kw, curvi in ((dict(grid="curvilinear", x=X, y=Y, **base), True), (base, False)):
        a = mdf.Solver(n, n, **kw)
        b = mdf.Solver(n, n, rho0=True, **kw)
        for s in (a, b):
            s.set_launch(*plan)
            s.init(*W.zeros(n, n))
        b.init_rho0(1 + 0.3 * np.random.default_rng(4).random((n, n)))
        a.step(200)
        b.step(200)
        if curvi or plan == (0, 0):
            np.testing.assert_array_equal(a.state(), b.state())
        else:
            assert maxabs(a.state(), b.state()) <= 1e-6 * U0


@pytest.mark.parametrize("plan", [(128, 3), (0, 0)])
@pytest.mark.parametrize("grid", ["uniform", "curvilinear"])
def test_both_kernel_families_against_oracle(plan, grid):
    """The lane on the shared-ring march and on the tile kernel: a power-law
    cavity with a source field and a rho_0 pattern, against the oracle."""
    n, U0 = 37, 0.1
    kw = dict(nu=0.004, walls=(True, True), u_wall=(0, 0, 0, U0), power_law=(0.004, 0.8, 2e-4, 0.08))
    if grid == "curvilinear":
        X, Y = W.trapezoid_grid(n, n)
        kw.update(grid="curvilinear", x=X, y=Y)
    g, o = both(n, n, **kw)
    g.set_launch(*plan)
    assert g.launch_info()["kernel"] == ("tile" if plan == (0, 0) else "march")
    Xn, Yn = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n))
    for s in (g, o):
        s.init(*W.zeros(n, n))
        s.init_rho0(1 + 0.1 * np.cos(np.pi * Xn) * np.sin(np.pi * Yn))
    g.step(300)
    o.step(300)
    check(g, o, U0)


def periodic_case(grid, forced, nx=300, ny=90, nu=0.01, u0=0.05):
    """The periodic flow of Sec. 4.2 on [0, 1) x [0, ny/nx), uniform or with
    smoothly stretched periodic y nodes; forced: its body force as a field,
    a constant force rate and a source field R."""
    ly = ny / nx
    kw = dict(nu=nu, lx=1.0, ly=ly)
    X, Y = np.meshgrid(W.periodic_nodes(nx, 1.0), W.periodic_nodes(ny, ly))
    if grid == "separable":
        j = np.arange(ny)
        y = ly * (j / ny + 0.02 * np.sin(2 * np.pi * j / ny) / (2 * np.pi))
        kw.update(grid="separable", x=W.periodic_nodes(nx, 1.0), y=y)
        X, Y = np.meshgrid(W.periodic_nodes(nx, 1.0), y)
    u, v, Fx, Fy = W.periodic_flow_at(X, Y / ly, u0, nu)
    if forced:
        kw.update(force=(Fx, Fy), force_rate=(2e-4, -1e-4),
                  source=0.01 * np.sin(2 * math.pi * X) * np.cos(2 * math.pi * Y / ly))
    rho = 1 + 0.1 * np.sin(2 * math.pi * X) * np.cos(2 * math.pi * Y / ly)
    return kw, u, v, rho


@pytest.mark.parametrize("forced", [False, True])
@pytest.mark.parametrize("grid", ["uniform", "separable"])
def test_periodic_register_march_against_oracle(grid, forced):
    """The lane on the periodic register-window march (128 threads): three
    strips of 120 columns (the last ragged) and bands of 37 rows (the last
    ragged), 300 steps against the oracle; forced adds a force field, a force
    rate and a source field to both streaming steps."""
    nx, ny, u0 = 300, 90, 0.05
    kw, u, v, rho = periodic_case(grid, forced, nx, ny, u0=u0)
    g, o = both(nx, ny, **kw)
    g.set_launch(128, 37)
    assert g.launch_info()["kernel"] == "march" and g.launch_info()["threads"] == 128
    z = np.zeros((ny, nx))
    for s in (g, o):
        if forced:
            s.init(z, z, z)
        else:
            s.init(u, v, z)
        s.init_rho0(rho)
    g.step(300)
    o.step(300)
    check(g, o, u0)


@pytest.mark.parametrize("forced", [False, True])
def test_no_feedback_on_the_periodic_register_march_bitwise(forced):
    """Remark 1 on the periodic register-window march: the same plan with and
    without the lane gives the alpha = 1, 2 state to the bit."""
    nx, ny = 300, 90
    kw, u, v, rho = periodic_case("uniform", forced, nx, ny)
    a = mdf.Solver(nx, ny, **kw)
    b = mdf.Solver(nx, ny, rho0=True, **kw)
    z = np.zeros((ny, nx))
    for s in (a, b):
        s.set_launch(128, 37)
        s.init(u, v, z)
    b.init_rho0(rho)
    a.step(200)
    b.step(200)
    np.testing.assert_array_equal(a.state(), b.state())


def test_state_roundtrip_and_checkpoint(tmp_path):
    n = 24
    g = mdf.Solver(n, n, nu=0.01, walls=(True, True), u_wall=(0, 0, 0, 0.1), rho0=True)
    g.init(*W.zeros(n, n))
    g.step(30)
    r = W.random_state(n, n, 0.01, 9)[0] + 0.2  # any 5 planes
    g.set_rho0_state(r.astype(np.float32))
    np.testing.assert_array_equal(g.rho0_state(), r.astype(np.float32))
    g.save(tmp_path / "r.ckpt")
    g.step(40)
    h = mdf.Solver(n, n, nu=0.01, walls=(True, True), u_wall=(0, 0, 0, 0.1), rho0=True)
    h.load(tmp_path / "r.ckpt")
    assert h.steps == 30
    h.step(40)
    np.testing.assert_array_equal(g.rho0_state(), h.rho0_state())
    np.testing.assert_array_equal(g.state(), h.state())
    # 10- and 15-plane checkpoints do not mix
    other = mdf.Solver(n, n, nu=0.01, walls=(True, True), u_wall=(0, 0, 0, 0.1))
    with pytest.raises(mdf.MdfError) as e:
        other.load(tmp_path / "r.ckpt")
    assert e.value.status == mdf.MDF_E_INVALID


def test_bytes_routing_and_rejections():
    g = mdf.Solver(64, 64, nu=0.01, rho0=True)
    assert g.bytes_per_node() == 120.0
    assert g.launch_info()["threads"] in (128, 256)
    plain = mdf.Solver(16, 16, nu=0.01)
    with pytest.raises(mdf.MdfError) as e:
        plain.rho0()
    assert e.value.status == mdf.MDF_E_INVALID
    with pytest.raises(mdf.MdfError) as e:
        mdf.Solver(16, 16, nu=0.01, storage="fp16", rho0=True)
    assert e.value.status == mdf.MDF_E_INVALID


def test_large_periodic_grid_sampled():
    """1024^2 Taylor-Green flow with a rho_0 pattern, several strips and
    bands per block row, against the oracle on the full grid (3 steps), in
    the plan the autotuner picks."""
    n, U0 = 1024, 0.01
    kw = dict(nu=0.01, lx=2 * math.pi, ly=2 * math.pi)
    g, o = both(n, n, **kw)
    X, Y = np.meshgrid(np.arange(n) / n, np.arange(n) / n)
    for s in (g, o):
        s.init(*W.taylor_green(n, U0))
        s.init_rho0(1 + 0.1 * np.sin(2 * math.pi * X) * np.cos(4 * math.pi * Y))
    g.step(3)
    o.step(3)
    check(g, o, U0)
