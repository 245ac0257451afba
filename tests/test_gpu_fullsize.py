"""Full-size parity of the benchmark workloads that have no other full-size
check: the power-law cavity on the 513 x 513 body-fitted trapezoid grid and
the seeded 512-cavity batched sweep, in the launch configurations the
benchmark times, against the FP64 oracle on the full grid (a few steps from
rest; the FP32 parity bar, 1e-5 times the lid speed)."""
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


def power_law_cavity(n_index, re, u0=U0):
    """K from Re = u0^(2-n) L^n / K with L = 1; nu clamped to [nu_ref/20, 20 nu_ref]."""
    K = u0 ** (2.0 - n_index) / re
    nu_ref = K * u0 ** (n_index - 1.0)
    return dict(nu=nu_ref, walls=(True, True), u_wall=(0, 0, 0, u0),
                power_law=(K, float(n_index), nu_ref / 20, nu_ref * 20))


@pytest.mark.parametrize("n_index,re", [(0.5, 1000.0), (1.5, 100.0)])
def test_trapezoid_513_power_law_against_oracle(n_index, re):
    n = 513
    X, Y = W.trapezoid_grid(n, n)
    kw = dict(grid="curvilinear", x=X, y=Y, **power_law_cavity(n_index, re))
    g, o = mdf.Solver(n, n, **kw), Oracle(n, n, **kw)
    for s in (g, o):
        s.init(*W.zeros(n, n))
    g.step(5)
    o.step(5)
    err = float(np.abs(g.state().astype(np.float64) - o.state()).max())
    assert err <= 1e-5 * U0, err


def test_512_cavity_batch_sample_against_oracle():
    """The seeded sweep (sides 65-513, Re 100-5000, n 0.5-1.5) stepped as one
    batch; the first problem of every side is checked against the oracle."""
    re, nn, sides = W.cavity_batch_draws(512, 2306)
    probs = [dict(nx=int(sd), ny=int(sd), **power_law_cavity(float(b), float(a))) for a, b, sd in zip(re, nn, sides)]
    batch = mdf.Batch(probs)
    batch.step(3)
    info = batch.info()
    assert info["problems"] == 512 and info["steps"] == 3
    checked = 0
    for side in (65, 129, 257, 513):
        i = int(np.nonzero(sides == side)[0][0])
        kw = dict(probs[i])
        nx, ny = kw.pop("nx"), kw.pop("ny")
        o = Oracle(nx, ny, **kw)
        o.init(*W.zeros(nx, ny))
        o.step(3)
        err = float(np.abs(batch.problem(i).state().astype(np.float64) - o.state()).max())
        assert err <= 1e-5 * U0, (side, err)
        checked += 1
    assert checked == 4
