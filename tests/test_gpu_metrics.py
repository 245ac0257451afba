"""GPU parity of the body-fitted path with metric coefficients given by the
caller (mdf_set_metrics) against the oracle given the same coefficients:
the exact derivatives of a non-affine doubly periodic map and of the
trapezoid map, on the shared-ring march and on the tile kernel.  The FP32
parity bar, 1e-5 of the reference velocity."""
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

PLANS = [(128, 7), (0, 0)]


def maxabs(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max())


@pytest.mark.parametrize("plan", PLANS)
def test_distorted_periodic_grid_with_exact_metrics(plan):
    """x = xi + a sin 2 pi eta, y = eta + a sin 2 pi xi (50^2, ragged against
    16-node tiles and 7-row bands), the periodic flow of Sec. 4.2 driven from
    rest for 300 steps.  The exact metrics differ from the differenced ones
    by O(h^2), which moves the state by about 2e-4 of the reference velocity
    here: the GPU run must match the oracle with the same given metrics to
    the parity bar and stay away from the oracle with differenced ones."""
    n, a, nu, u0 = 50, 0.06, 0.01, 0.05
    X, Y = W.distorted_periodic_grid(n, a)
    u, v, Fx, Fy = W.periodic_flow_at(X, Y, u0, nu)
    kw = dict(nu=nu, grid="curvilinear", x=X, y=Y, lx=1.0, ly=1.0, force=(Fx, Fy))
    g, o, od = mdf.Solver(n, n, **kw), Oracle(n, n, **kw), Oracle(n, n, **kw)
    m = W.distorted_periodic_metrics(n, a)
    g.set_metrics(*m)
    o.set_metrics(*m)
    g.set_launch(*plan)
    assert g.launch_info()["kernel"] == ("tile" if plan == (0, 0) else "march")
    z = np.zeros((n, n))
    for s in (g, o, od):
        s.init(z, z, z)
    g.step(300)
    o.step(300)
    od.step(300)
    assert maxabs(g.state(), o.state()) <= 1e-5 * u0
    assert maxabs(g.state(), od.state()) >= 5e-5 * u0


@pytest.mark.parametrize("plan", PLANS)
def test_trapezoid_cavity_with_exact_metrics(plan):
    """The lid-driven trapezoid cavity (walls on both axes) with the exact
    metrics of the bilinear map passed in, against the oracle given the
    same: the wall columns, ghost zeros and corner nodes of the given-metric
    path."""
    n, u0 = 41, 0.1
    X, Y = W.trapezoid_grid(n, n)
    kw = dict(nu=0.01, grid="curvilinear", x=X, y=Y, walls=(True, True), u_wall=(0, 0, 0, u0))
    g, o = mdf.Solver(n, n, **kw), Oracle(n, n, **kw)
    m = W.trapezoid_metrics(n, n)
    g.set_metrics(*m)
    o.set_metrics(*m)
    g.set_launch(*plan)
    z = np.zeros((n, n))
    for s in (g, o):
        s.init(z, z, z)
    g.step(400)
    o.step(400)
    assert maxabs(g.state(), o.state()) <= 1e-5 * u0


def test_set_metrics_rejections():
    g = mdf.Solver(16, 16, nu=0.01)
    one = np.ones((16, 16))
    with pytest.raises(mdf.MdfError) as e:
        g.set_metrics(one, 0 * one, 0 * one, one)
    assert e.value.status == mdf.MDF_E_INVALID
    X, Y = W.distorted_periodic_grid(16, 0.05)
    h = mdf.Solver(16, 16, nu=0.01, grid="curvilinear", x=X, y=Y, lx=1.0, ly=1.0)
    bad = W.distorted_periodic_metrics(16, 0.05)
    bad[0][3, 4] = np.nan
    with pytest.raises(mdf.MdfError) as e:
        h.set_metrics(*bad)
    assert e.value.status == mdf.MDF_E_INVALID
