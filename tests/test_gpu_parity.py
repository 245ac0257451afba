"""GPU parity: the fused CUDA step (through the C ABI) against the FP64 oracle.

Every case feeds both sides the same seeded inputs from
paper_2306_08216_gb300.workloads and compares element by element.  The
tolerance is the one the work is held to: max |GPU - oracle| <= 1e-5 times the
reference velocity after the stated number of steps (FP32 state and
arithmetic against FP64; the scheme is dissipative, so FP32 rounding stays
bounded).  Short runs on tiny and ragged grids use a tighter bound.
"""
import math

import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_2306_08216_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect with -m "not gpu"
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2306_08216_gb300 import build as B  # noqa: E402
from paper_2306_08216_gb300 import mdf  # noqa: E402

B.build()


def pair(nx, ny, **kw):
    return mdf.Solver(nx, ny, **kw), Oracle(nx, ny, **kw)


def run_both(g, o, fields, steps):
    g.init(*fields)
    o.init(*fields)
    g.step(steps)
    o.step(steps)
    g.synchronize()
    return g.state().astype(np.float64), o.state()


def maxabs(a, b):
    return float(np.abs(a - b).max())


# ------------------------------------------------------------ spec case


def test_taylor_green_64_after_1000_steps():
    """64^2, U0 = 0.01, nu = 0.01, CFL 0.5, 1000 steps: max abs <= 1e-5 U0."""
    n, U0 = 64, 0.01
    g, o = pair(n, n, nu=0.01, lx=2 * math.pi, ly=2 * math.pi)
    sg, so = run_both(g, o, W.taylor_green(n, U0), 1000)
    assert maxabs(sg, so) <= 1e-5 * U0
    fg, fo = g.fields(), o.fields()
    for k in ("u", "v"):
        assert maxabs(fg[k], fo[k]) <= 1e-5 * U0


# --------------------------------------------- tiny, ragged and multi-tile grids


@pytest.mark.parametrize("nx,ny", [(5, 5), (12, 9), (31, 17), (121, 11), (130, 7), (247, 13), (250, 40)])
@pytest.mark.parametrize("walls", [(False, False), (True, True), (False, True), (True, False)])
def test_small_and_ragged_grids(nx, ny, walls):
    if walls[0] and nx < 5 or walls[1] and ny < 5:
        pytest.skip("too small")
    U = 0.05
    kw = dict(nu=0.004, lx=1.0, ly=0.8, walls=walls, u_wall=(0.0, 0.01, -0.02, U), v_wall=(0.02, 0.0, 0.0, -0.01),
              eta=0.7)
    g, o = pair(nx, ny, **kw)
    u, v, p = W.random_fields(nx, ny, U, seed=nx * 131 + ny)
    sg, so = run_both(g, o, (u, v, p), 6)
    assert maxabs(sg, so) <= 2e-6 * U


def test_zero_and_negative_step_counts():
    """mdf_step(0) changes nothing and mdf_step(-1) is MDF_E_INVALID with the
    state untouched; a batch behaves the same."""
    g = mdf.Solver(20, 20, nu=0.01, walls=(True, True), u_wall=(0, 0, 0, 0.1))
    g.init(*W.zeros(20, 20))
    g.step(7)
    s0 = g.state()
    g.step(0)
    np.testing.assert_array_equal(g.state(), s0)
    with pytest.raises(mdf.MdfError) as e:
        g.step(-1)
    assert e.value.status == mdf.MDF_E_INVALID
    np.testing.assert_array_equal(g.state(), s0)
    assert g.steps == 7
    b = mdf.Batch([dict(nx=20, ny=20, nu=0.01, walls=(True, True), u_wall=(0, 0, 0, 0.1))])
    b.step(3)
    t0 = b.problem(0).state()
    b.step(0)
    np.testing.assert_array_equal(b.problem(0).state(), t0)
    with pytest.raises(mdf.MdfError):
        b.step(-2)
    assert b.info()["steps"] == 3


def test_set_state_roundtrip_and_single_step():
    nx, ny = 70, 33
    g, o = pair(nx, ny, nu=0.01, lx=1.3, ly=1.0)
    fh = W.random_state(nx, ny, 0.01, seed=3)
    g.set_state(fh)
    np.testing.assert_array_equal(g.state(), fh.astype(np.float32))
    o.set_state(fh.astype(np.float32).astype(np.float64))
    g.step(1)
    o.step(1)
    assert maxabs(g.state().astype(np.float64), o.state()) <= 2e-8


@pytest.mark.parametrize("threads,rows", [(128, 8), (128, 37), (256, 8), (256, 64), (128, 1), (128, 3), (256, 2)])
def test_launch_plans_agree_with_oracle(threads, rows):
    """Every block size / band height the autotuner may pick (periodic fast
    path): ragged strips and bands against the oracle."""
    nx, ny = 300, 150
    u, v, p = W.random_fields(nx, ny, 0.05, seed=17)
    g, o = pair(nx, ny, nu=0.004, lx=1.0, ly=0.6)
    g.set_launch(threads, rows)
    sg, so = run_both(g, o, (u, v, p), 20)
    assert maxabs(sg, so) <= 2e-6 * 0.05


# ---------------------------------------------------------- walls and forces


def test_lid_driven_cavity_33_after_1000_steps():
    n, u0 = 33, 0.1
    kw = dict(nu=0.1 / 100.0, walls=(True, True), u_wall=(0, 0, 0, u0))
    g, o = pair(n, n, **kw)
    sg, so = run_both(g, o, W.zeros(n, n), 1000)
    assert maxabs(sg, so) <= 1e-5 * u0
    fg, fo = g.fields(), o.fields()
    assert maxabs(fg["u"], fo["u"]) <= 1e-5 * u0
    assert np.abs(fg["u"][-1, 1:-1] - u0).max() <= 1e-6 * u0


def test_poiseuille_constant_force():
    n, F, nu = 32, 1e-4, 0.01
    kw = dict(nu=nu, walls=(False, True), force=(F, 0.0))
    g, o = pair(n, n, **kw)
    sg, so = run_both(g, o, W.zeros(n, n), 1000)
    umax = F / (8 * nu)
    assert maxabs(sg, so) <= 1e-5 * umax


def test_periodic_flow_force_field_anisotropic():
    nx, ny, nu, u0 = 64, 32, 0.01, 0.05
    u, v, p, Fx, Fy, _ = W.periodic_flow(nx, ny, u0=u0, nu=nu)
    kw = dict(nu=nu, force=(Fx, Fy))
    g, o = pair(nx, ny, **kw)
    sg, so = run_both(g, o, W.zeros(nx, ny), 500)
    assert maxabs(sg, so) <= 1e-5 * u0


# ------------------------------------------------- grids: separable, curvilinear


def test_tanh_stretched_cavity():
    n, u0 = 41, 0.1
    xs = W.tanh_nodes(n, 1.5)
    kw = dict(nu=0.1 / 100.0, grid="separable", x=xs, y=xs, walls=(True, True), u_wall=(0, 0, 0, u0))
    g, o = pair(n, n, **kw)
    assert abs(g.dt - o.dt) <= 1e-12 * o.dt
    sg, so = run_both(g, o, W.zeros(n, n), 600)
    assert maxabs(sg, so) <= 1e-5 * u0


def test_trapezoid_cavity_curvilinear():
    nx, ny, u0 = 37, 29, 0.1
    X, Y = W.trapezoid_grid(nx, ny)
    kw = dict(nu=0.1 / 100.0, grid="curvilinear", x=X, y=Y, walls=(True, True), u_wall=(0, 0, 0, u0))
    g, o = pair(nx, ny, **kw)
    assert abs(g.dt - o.dt) <= 1e-12 * o.dt
    sg, so = run_both(g, o, W.zeros(nx, ny), 400)
    assert maxabs(sg, so) <= 1e-5 * u0


def test_separable_periodic_channel():
    nx, ny = 24, 33
    kw = dict(nu=0.01, grid="separable", x=W.periodic_nodes(nx, 1.0), y=W.tanh_nodes(ny, 1.5), lx=1.0,
              walls=(False, True), force=(1e-4, 0.0))
    g, o = pair(nx, ny, **kw)
    sg, so = run_both(g, o, W.zeros(nx, ny), 300)
    assert maxabs(sg, so) <= 1e-5 * (1e-4 / (8 * 0.01))


def test_separable_periodic_stretched_axis_with_force_field():
    """Both axes periodic, y nodes smoothly stretched (periodic metric
    continuation across the seam), forcing-field variant of the fast path."""
    nx, ny, nu, u0 = 48, 40, 0.01, 0.05
    j = np.arange(ny)
    y = j / ny + 0.02 * np.sin(2 * np.pi * j / ny) / (2 * np.pi)
    _, _, _, Fx, Fy, _ = W.periodic_flow(nx, ny, u0=u0, nu=nu)
    kw = dict(nu=nu, grid="separable", x=W.periodic_nodes(nx, 1.0), y=y, lx=1.0, ly=1.0, force=(Fx, Fy))
    g, o = pair(nx, ny, **kw)
    sg, so = run_both(g, o, W.zeros(nx, ny), 500)
    assert maxabs(sg, so) <= 1e-5 * u0


# ---------------------------------------------------------------- power law


@pytest.mark.parametrize("n_index", [0.5, 1.0, 1.5])
def test_power_law_cavity(n_index):
    n, u0 = 33, 0.1
    K = 0.1 * 0.1 ** (n_index - 1) / 100.0  # Re = u0^(2-n) L^n / K = 100
    kw = dict(nu=K, walls=(True, True), u_wall=(0, 0, 0, u0), power_law=(K, n_index, K / 20, K * 20))
    g, o = pair(n, n, **kw)
    sg, so = run_both(g, o, W.zeros(n, n), 500)
    assert maxabs(sg, so) <= 1e-5 * u0
    fg, fo = g.fields(["nu"]), o.fields()
    np.testing.assert_allclose(fg["nu"], fo["nu"], rtol=2e-3)


# ----------------------------------------------------------- derived fields


def test_derived_fields_match_oracle():
    nx, ny, nu = 48, 40, 0.01
    u, v, p, Fx, Fy, _ = W.periodic_flow(nx, ny, u0=0.05, nu=nu)
    kw = dict(nu=nu, force=(Fx, Fy))
    g, o = pair(nx, ny, **kw)
    run_both(g, o, (u, v, p), 200)
    fg, fo = g.fields(), o.fields()
    grad = max(np.abs(fo[k]).max() for k in ("dudx", "dudy", "dvdx", "dvdy"))
    scale = {k: grad for k in ("dudx", "dudy", "dvdx", "dvdy", "div", "Sxx", "Sxy", "Syy", "Omega_xy", "vorticity")}
    scale.update({k: 2 * nu * grad for k in ("sigma_xx", "sigma_xy", "sigma_yy")})
    for k in mdf.FIELD_NAMES:
        sc = scale.get(k, np.abs(fo[k]).max())
        assert maxabs(fg[k], fo[k]) <= 2e-4 * sc, k


def test_fields_into_caller_arrays():
    """fields(out=...) writes into the caller's host arrays (numpy, or CPU
    torch tensors in pinned memory) the same bits fields() returns; a
    wrong shape or dtype is refused before any copy."""
    nx, ny = 37, 29
    g = mdf.Solver(nx, ny, nu=0.01, walls=(True, True), u_wall=(0, 0, 0, 0.1))
    g.init(*W.random_fields(nx, ny, 0.02, 3))
    g.step(40)
    ref = g.fields(["u", "v", "P", "vorticity"])
    pinned = {k: torch.empty((ny, nx), dtype=torch.float32).pin_memory() for k in ("u", "P")}
    plain = {"v": np.zeros((ny, nx), np.float32)}
    got = g.fields(["u", "v", "P", "vorticity"], out={**pinned, **plain})
    assert got["u"] is pinned["u"] and got["v"] is plain["v"]
    for k in ("u", "v", "P", "vorticity"):
        np.testing.assert_array_equal(np.asarray(got[k]), ref[k])
    with pytest.raises(AssertionError):
        g.fields(["u"], out={"u": np.zeros((nx, ny), np.float32)})
    with pytest.raises(AssertionError):
        g.fields(["u"], out={"u": np.zeros((ny, nx), np.float64)})


# --------------------------------------------------------- residual & drift


def test_residual_and_drift_follow_their_definition():
    n, U0, K = 64, 0.01, 50
    g, o = pair(n, n, nu=0.01, lx=2 * math.pi, ly=2 * math.pi)
    fields = W.taylor_green(n, U0)
    g.init(*fields)
    o.init(*fields)
    u0, v0 = o.fields()["u"], o.fields()["v"]
    g.step(K)
    o.step(K)
    r, drift = g.residual()
    fo = o.fields()
    num = math.sqrt(((fo["u"] - u0) ** 2 + (fo["v"] - v0) ** 2).sum())
    den = math.sqrt((fo["u"] ** 2 + fo["v"] ** 2).sum())
    assert r == pytest.approx(num / (K * den), rel=1e-4)
    tol = 1e-6 * np.abs(fo["u"]).sum()
    assert abs(drift[0] - fo["u"].sum()) <= tol and abs(drift[1] - fo["v"].sum()) <= tol
    with pytest.raises(mdf.MdfError) as e:
        g.residual()  # no step since the snapshot
    assert e.value.status == mdf.MDF_E_STATE


def test_residual_in_two_halves_equals_the_synchronous_residual():
    """mdf_residual_start / _finish with steps enqueued in between return the
    residual and drift of the state at the start, equal to the bit to
    mdf_residual on a twin run; the next window is measured from that
    snapshot; a second start or a finish with none pending is MDF_E_STATE."""
    n = 33
    kw = dict(nu=0.01, walls=(True, True), u_wall=(0, 0, 0, 0.1))
    a, b = mdf.Solver(n, n, **kw), mdf.Solver(n, n, **kw)
    for s in (a, b):
        s.init(*W.zeros(n, n))
        s.step(50)
    ra = a.residual()
    b.residual_start()
    with pytest.raises(mdf.MdfError) as e:
        b.residual_start()
    assert e.value.status == mdf.MDF_E_STATE
    b.step(50)
    rb = b.residual_finish()
    assert ra == rb
    a.step(50)
    assert a.residual() == b.residual()
    with pytest.raises(mdf.MdfError) as e:
        b.residual_finish()
    assert e.value.status == mdf.MDF_E_STATE


def test_divergence_is_reported():
    """Table 2: nu = 1e-3, F = 0.1 on 32 x 32 diverges; the library reports it."""
    n = 32
    g = mdf.Solver(n, n, nu=1e-3, walls=(False, True), force=(0.1, 0.0))
    g.init(*W.zeros(n, n))
    status = None
    for _ in range(40):
        g.step(250)
        try:
            g.residual()
        except mdf.MdfError as e:
            status = e.status
            break
    assert status == mdf.MDF_E_DIVERGED


# ------------------------------------------------------------- checkpoints


def test_checkpoint_resume_is_bitwise(tmp_path):
    n = 40
    kw = dict(nu=0.002, walls=(True, True), u_wall=(0, 0, 0, 0.1))
    a = mdf.Solver(n, n, **kw)
    a.init(*W.zeros(n, n))
    a.step(30)
    a.save(tmp_path / "c.ckpt")
    a.step(20)
    b = mdf.Solver(n, n, **kw)
    b.load(tmp_path / "c.ckpt")
    assert b.steps == 30
    b.step(20)
    np.testing.assert_array_equal(a.state(), b.state())


# ------------------------------------------------ device pointers and streams


def test_device_inputs_outputs_and_stream():
    n, U0 = 96, 0.01
    s = torch.cuda.Stream()
    g = mdf.Solver(n, n, nu=0.01, lx=2 * math.pi, ly=2 * math.pi, stream=s)
    u, v, p = W.taylor_green(n, U0)
    dev = [torch.tensor(t, dtype=torch.float32, device="cuda") for t in (u, v, p)]
    torch.cuda.synchronize()
    g.init(*dev)
    g.step(10)
    out = {k: torch.empty((n, n), dtype=torch.float32, device="cuda") for k in ("u", "v")}
    g.fields_device(out)
    st = torch.empty((2, 5, n, n), dtype=torch.float32, device="cuda")
    g.state(out=st)
    g.synchronize()
    h = mdf.Solver(n, n, nu=0.01, lx=2 * math.pi, ly=2 * math.pi)
    h.init(u, v, p)
    h.step(10)
    np.testing.assert_array_equal(st.cpu().numpy(), h.state())
    np.testing.assert_array_equal(out["u"].cpu().numpy(), h.fields(["u"])["u"])


# ----------------------------------------- full size, bench launch configuration


def test_taylor_green_4096_full_size_against_oracle():
    """The benchmark workload (4096^2, bench launch plan): three steps against
    the oracle on the full grid, then properties over 200 steps (momentum is
    conserved, the amplitude decays as exp(-2 nu t))."""
    n, U0, nu = 4096, 0.01, 0.01
    u, v, p = W.taylor_green(n, U0)
    g = mdf.Solver(n, n, nu=nu, lx=2 * math.pi, ly=2 * math.pi)
    o = Oracle(n, n, nu=nu, lx=2 * math.pi, ly=2 * math.pi)
    sg, so = run_both(g, o, (u, v, p), 3)
    assert maxabs(sg, so) <= 5e-7 * U0  # a few FP32 ulps of the largest fhat (~U0/5)
    del o, so, sg
    g.init(u, v, p)
    g.step(200)
    r, drift = g.residual()
    f = g.fields(["u"])
    t = 200 * g.dt
    amp = float((f["u"].astype(np.float64) * u).sum() / (u * u).sum())
    # the initial layer of an equilibrium start shifts the amplitude by ~5e-4
    assert abs(amp - math.exp(-2 * nu * t)) < 1e-3
    assert abs(drift[0]) < 1e-6 * n * n * U0 and abs(drift[1]) < 1e-6 * n * n * U0


def test_16384_grid_beyond_32_bit_offsets_equals_the_tiled_64_grid():
    """Maximum-size indexing: a 16384^2 periodic grid (10 planes of 269 M
    floats, so plane offsets pass 2^31 elements) started from a 64^2
    Taylor-Green period tiled 256 x 256 times.  The scheme is translation
    invariant, so after 40 steps every 64^2 block of every distribution
    plane must equal the oracle's solution of one period (same dx, dt) to the
    parity bar (compared on the device); the momentum drift stays zero and
    the residual finite."""
    n, m, U0, nu = 16384, 64, 0.01, 0.01
    L = 2 * math.pi
    u, v, p = W.taylor_green(m, U0, length=L * m / n)
    g = mdf.Solver(n, n, nu=nu, lx=L, ly=L)
    assert g.launch_info()["kernel"] == "march"
    g.init(*(np.tile(a.astype(np.float32), (n // m, n // m)) for a in (u, v, p)))
    o = Oracle(m, m, nu=nu, lx=L * m / n, ly=L * m / n)
    o.init(u, v, p)
    assert abs(g.dt - o.dt) <= 1e-12 * o.dt
    g.step(40)
    o.step(40)
    st = torch.empty((2, 5, n, n), dtype=torch.float32, device="cuda")
    g.state(out=st)
    g.synchronize()
    ref = torch.tensor(o.state(), dtype=torch.float64, device="cuda")
    err = 0.0
    for a in range(2):
        for j in range(5):
            blocks = st[a, j].view(n // m, m, n // m, m).double()
            err = max(err, float((blocks - ref[a, j][None, :, None, :]).abs().max()))
            del blocks
    del st
    assert err <= 1e-5 * U0, err
    r, drift = g.residual()
    assert np.isfinite(r) and abs(drift[0]) < 1e-6 * n * n * U0 and abs(drift[1]) < 1e-6 * n * n * U0


def test_graph_replay_equals_single_launches():
    """mdf_step(n >= 32) replays captured graphs of 16 launches; the result is
    bitwise the same as n single launches, and a force or launch-plan change
    between calls takes effect (the graphs are rebuilt)."""
    n = 48
    kw = dict(nu=0.01, walls=(False, True), force=(1e-4, 0.0))
    a, b = mdf.Solver(n, n, **kw), mdf.Solver(n, n, **kw)
    for s in (a, b):
        s.set_launch(0)  # the tile kernel first, a march below
        s.init(*W.zeros(n, n))
    a.step(70)                      # 4 graph replays + 6 launches
    for _ in range(70):
        b.step(1)
    np.testing.assert_array_equal(a.state(), b.state())
    for s in (a, b):
        s.set_force((2e-4, 1e-5))
    a.step(33)                      # odd start parity after 70 + 33 ...
    a.step(64)
    for _ in range(97):
        b.step(1)
    np.testing.assert_array_equal(a.state(), b.state())
    a.set_launch(256, 8)
    b.set_launch(256, 8)
    a.step(48)
    for _ in range(48):
        b.step(1)
    np.testing.assert_array_equal(a.state(), b.state())
    assert a.steps == b.steps == 215


@pytest.mark.parametrize("threads,rows", [(128, 2), (128, 5), (256, 3), (128, 8)])
def test_wall_kernel_launch_plans_agree_with_oracle(threads, rows):
    """Band heights down to a couple of rows on the wall and power-law
    kernel: a power-law cavity and a channel against the oracle."""
    n = 45
    kw = dict(nu=0.004, walls=(True, True), u_wall=(0, 0, 0, 0.1), power_law=(0.004, 0.8, 2e-4, 0.08))
    g, o = pair(n, n, **kw)
    g.set_launch(threads, rows)
    sg, so = run_both(g, o, W.zeros(n, n), 60)
    assert maxabs(sg, so) <= 1e-5 * 0.1
    kw = dict(nu=0.01, walls=(False, True), force=(1e-4, 0.0))
    g, o = pair(70, 33, **kw)
    g.set_launch(threads, rows)
    sg, so = run_both(g, o, W.zeros(70, 33), 60)
    assert maxabs(sg, so) <= 1e-5 * (1e-4 / (8 * 0.01))
