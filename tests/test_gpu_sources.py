"""GPU parity of the continuity source R (Eq. 2.3.23) and the dF/dt term
(Eq. 2.3.24) against the FP64 oracle, on the periodic fast path and on the
general (wall) kernel.  Tolerance: the FP32 parity bar, max |GPU - oracle|
<= 1e-5 times the reference velocity."""
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


def manufactured(nx, ny, nu, U0=0.05, a=0.02):
    """u = U0 + a sin(2 pi x), v = 0, R = u_x, F_x = d(u^2)/dx - nu u_xx."""
    k = 2 * math.pi
    X = np.tile(np.arange(nx) / nx, (ny, 1))
    u = U0 + a * np.sin(k * X)
    ux, uxx = a * k * np.cos(k * X), -a * k * k * np.sin(k * X)
    return u, ux, 2 * u * ux - nu * uxx


@pytest.mark.parametrize("c", [1.0, 2.0])
def test_source_field_on_the_fast_path(c):
    nx, ny, nu, U0 = 32, 8, 0.01, 0.05
    u, R, Fx = manufactured(nx, ny, nu, U0)
    kw = dict(nu=nu, lx=1.0, ly=ny / nx, c=c, force=(Fx, 0 * Fx), source=R)
    g, o = mdf.Solver(nx, ny, **kw), Oracle(nx, ny, **kw)
    for s in (g, o):
        s.init(u, 0 * u, 0 * u)
    g.step(1000)  # the parity window; the steady state itself is pinned on the oracle
    o.step(1000)
    assert maxabs(g.state(), o.state()) <= 1e-5 * U0
    fg, fo = g.fields(["u", "P", "div"]), o.fields()
    assert maxabs(fg["u"], fo["u"]) <= 1e-5 * U0
    assert maxabs(fg["P"], fo["P"]) <= 1e-5 * U0
    # the library's divergence (first-moment) follows R
    assert maxabs(fg["div"], R) <= 1e-3 * np.abs(R).max()


def test_constant_source_and_bytes():
    n = 24
    u, v, p = W.random_fields(n, n, 0.02, 5)
    kw = dict(nu=0.02, lx=1.0, ly=1.0, source=0.01)
    g, o = mdf.Solver(n, n, **kw), Oracle(n, n, **kw)
    for s in (g, o):
        s.init(u, v, p)
    g.step(200)
    o.step(200)
    assert maxabs(g.state(), o.state()) <= 1e-5 * 0.02
    h = mdf.Solver(n, n, nu=0.02, source=np.zeros((n, n)))
    assert h.bytes_per_node() == 84.0


def test_source_on_the_wall_kernel():
    """A smooth source field in a lid-driven cavity (walls, general kernel)."""
    n, U0 = 33, 0.1
    X, Y = np.meshgrid(np.linspace(0, 1, n), np.linspace(0, 1, n))
    R = 0.02 * np.sin(2 * np.pi * X) * np.sin(np.pi * Y)
    kw = dict(nu=0.01, walls=(True, True), u_wall=(0, 0, 0, U0), source=R)
    g, o = mdf.Solver(n, n, **kw), Oracle(n, n, **kw)
    for s in (g, o):
        s.init(*W.zeros(n, n))
    g.step(400)
    o.step(400)
    assert maxabs(g.state(), o.state()) <= 1e-5 * U0


@pytest.mark.parametrize("cfl", [0.4, 0.1])
def test_time_dependent_force_with_rate(cfl):
    """F_x = F0 cos(w t) set every step with its rate; uniform periodic flow."""
    n, F0, T = 8, 1e-3, 2.0
    w = 2 * math.pi / T
    g, o = mdf.Solver(n, n, nu=0.01, cfl=cfl), Oracle(n, n, nu=0.01, cfl=cfl)
    for s in (g, o):
        s.init(*W.zeros(n, n))
    steps = int(round(0.75 * T / o.dt))
    for k in range(steps):
        t = k * o.dt
        for s in (g, o):
            s.set_force((F0 * math.cos(w * t), 0.0))
            s.set_force_rate((-F0 * w * math.sin(w * t), 0.0))
            s.step(1)
    ug, uo = g.fields(["u"])["u"], o.fields()["u"]
    assert maxabs(ug, uo) <= 1e-5 * F0 / w
    exact = F0 / w * math.sin(w * steps * o.dt)
    assert abs(float(ug.mean()) - exact) < 1e-2 * F0 / w


@pytest.mark.parametrize("walls", [(False, False), (False, True)])
def test_force_and_rate_fields(walls):
    """Field force and field rate, changed every 20 steps, on the fast path
    (periodic) and on the wall kernel (channel)."""
    nx, ny, nu = 40, 24, 0.02
    X, Y = np.meshgrid(np.arange(nx) / nx, np.arange(ny) / ny)
    g = mdf.Solver(nx, ny, nu=nu, walls=walls)
    o = Oracle(nx, ny, nu=nu, walls=walls)
    for s in (g, o):
        s.init(*W.zeros(nx, ny))
    for block in range(5):
        a = 1e-4 * (1 + block)
        F = (a * np.sin(2 * np.pi * Y), 0.5 * a * np.cos(2 * np.pi * X))
        dF = (-0.1 * a * np.cos(2 * np.pi * X), 0.2 * a * np.sin(2 * np.pi * Y))
        for s in (g, o):
            s.set_force(F)
            s.set_force_rate(dF)
            s.step(20)
    ref = 1e-4 * 5 / (nu * (2 * np.pi) ** 2)  # velocity scale of the forcing
    assert maxabs(g.state(), o.state()) <= 1e-5 * ref


def test_source_is_rejected_where_it_is_not_defined():
    pl = mdf.Solver(16, 16, nu=0.01, power_law=(0.01, 0.8, 1e-4, 1.0), walls=(True, True))
    with pytest.raises(mdf.MdfError) as e:
        pl.set_source(0.1)
    assert e.value.status == mdf.MDF_E_INVALID
    s16 = mdf.Solver(16, 16, nu=0.01, storage="fp16")
    with pytest.raises(mdf.MdfError) as e:
        s16.set_source(0.1)
    assert e.value.status == mdf.MDF_E_INVALID
