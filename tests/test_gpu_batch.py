"""Batched step (one persistent launch per time step for many problems)
against the single-problem path and the oracle."""
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


def cavity(n, re, n_index=None, u0=0.1, m=None):
    m = n if m is None else m
    kw = dict(nx=n, ny=m, walls=(True, True), u_wall=(0, 0, 0, u0))
    if n_index is None:
        kw["nu"] = u0 / re
    else:
        K = u0 ** (2 - n_index) / re  # Re = u0^(2-n) L^n / K with L = 1
        kw["nu"] = K
        kw["power_law"] = (K, n_index, K / 20, K * 20)
    return kw


# the single-problem plan each batch kernel shares its values with (the
# rolled march computes what the unrolled one does)
SOLO_PLAN = {"march": (128, 8), "march_rolled": (128, 8), "tile": (0, 0)}


@pytest.mark.parametrize("kernel", ["march", "march_rolled", "tile"])
def test_batch_of_power_law_cavities_equals_solo_runs_bitwise(kernel):
    probs = [cavity(65, 400, 0.6), cavity(33, 100, 1.0), cavity(47, 250, 1.4, m=39), cavity(130, 1000, 0.9)]
    batch = mdf.Batch(probs)
    batch.set_launch(kernel)
    batch.step(40)   # graph replays (2 x 16) + 8 direct launches
    batch.step(3)
    for i, kw in enumerate(probs):
        kw = dict(kw)
        nx, ny = kw.pop("nx"), kw.pop("ny")
        solo = mdf.Solver(nx, ny, **kw)
        solo.set_launch(*SOLO_PLAN[kernel])
        solo.init(*W.zeros(nx, ny))
        solo.step(43)
        np.testing.assert_array_equal(batch.problem(i).state(), solo.state())
    info = batch.info()
    assert info["problems"] == 4 and info["steps"] == 43 and info["kernel"] == kernel


def test_batch_problem_against_oracle():
    probs = [cavity(41, 200), cavity(29, 150, m=35)]
    batch = mdf.Batch(probs)
    batch.step(300)
    for i, kw in enumerate(probs):
        kw = dict(kw)
        nx, ny = kw.pop("nx"), kw.pop("ny")
        o = Oracle(nx, ny, **kw)
        o.init(*W.zeros(nx, ny))
        o.step(300)
        assert np.abs(batch.problem(i).state().astype(np.float64) - o.state()).max() <= 1e-5 * 0.1


def test_batch_initial_fields_and_periodic_problems():
    n = 48
    probs = [dict(nx=n, ny=n, nu=0.01, lx=2 * math.pi, ly=2 * math.pi),
             dict(nx=70, ny=30, nu=0.005, lx=1.0, ly=0.5)]
    batch = mdf.Batch(probs)
    f0 = W.taylor_green(n, 0.01)
    f1 = W.random_fields(70, 30, 0.02, seed=4)
    batch.init(0, *f0)
    batch.init(1, *f1)
    batch.step(50)
    for i, (kw, f) in enumerate(zip(probs, (f0, f1))):
        kw = dict(kw)
        nx, ny = kw.pop("nx"), kw.pop("ny")
        o = Oracle(nx, ny, **kw)
        o.init(*f)
        o.step(50)
        assert np.abs(batch.problem(i).state().astype(np.float64) - o.state()).max() <= 2e-7


def test_batch_reports_divergence_per_problem():
    probs = [dict(nx=32, ny=32, nu=1e-3, walls=(False, True)),
             dict(nx=32, ny=32, nu=1e-2, walls=(False, True))]
    batch = mdf.Batch(probs)
    batch.problem(0).set_force((0.1, 0.0))   # Table 2: diverges at nu = 1e-3, F = 0.1
    batch.problem(1).set_force((1e-4, 0.0))
    status = None
    for _ in range(40):
        batch.step(250)
        r, status = batch.residual()
        if status[0] == mdf.MDF_E_DIVERGED:
            break
    assert status[0] == mdf.MDF_E_DIVERGED
    assert status[1] == mdf.MDF_OK and np.isfinite(r[1])


def test_batch_rejects_mixed_kernel_variants():
    with pytest.raises(mdf.MdfError) as e:
        mdf.Batch([cavity(33, 100), cavity(33, 100, 0.7)])
    assert e.value.status == mdf.MDF_E_INVALID


def _solo_state(kw, steps, kernel):
    kw = dict(kw)
    nx, ny = kw.pop("nx"), kw.pop("ny")
    solo = mdf.Solver(nx, ny, **kw)
    solo.set_launch(*SOLO_PLAN[kernel])
    solo.init(*W.zeros(nx, ny))
    solo.step(steps)
    return solo.state()


@pytest.mark.parametrize("kernel", ["march", "march_rolled", "tile"])
def test_retired_problems_freeze_and_resume_bitwise(kernel):
    """A retired problem keeps its state while the others advance; re-admitted
    after an odd number of batch steps (its buffers swap roles), it continues
    exactly as if it had been stepped alone."""
    probs = [cavity(65, 400, 0.8), cavity(40, 100, 1.2), cavity(33, 250, 1.0)]
    batch = mdf.Batch(probs)
    batch.set_launch(kernel)
    _solo = lambda kw, steps: _solo_state(kw, steps, kernel)  # noqa: E731
    batch.step(20)
    batch.set_active(1, False)
    batch.step(37)  # odd: the batch parity now differs from problem 1's
    r, st = batch.residual()
    assert st[1] == mdf.MDF_E_STATE and np.isnan(r[1])
    assert st[0] == mdf.MDF_OK and st[2] == mdf.MDF_OK
    np.testing.assert_array_equal(batch.problem(1).state(), _solo(probs[1], 20))
    np.testing.assert_array_equal(batch.problem(0).state(), _solo(probs[0], 57))
    batch.set_active(1, True)
    batch.step(35)
    np.testing.assert_array_equal(batch.problem(1).state(), _solo(probs[1], 55))
    np.testing.assert_array_equal(batch.problem(2).state(), _solo(probs[2], 92))
    assert batch.problem(1).steps == 55 and batch.problem(2).steps == 92
    for i in range(3):
        batch.set_active(i, False)
    batch.step(10)  # nothing left to step
    np.testing.assert_array_equal(batch.problem(2).state(), _solo(probs[2], 92))


def test_rolled_march_rejected_on_curvilinear_batches():
    X, Y = W.trapezoid_grid(33, 33)
    batch = mdf.Batch([dict(nx=33, ny=33, nu=0.01, grid="curvilinear", x=X, y=Y, walls=(True, True),
                            u_wall=(0, 0, 0, 0.1))])
    with pytest.raises(mdf.MdfError) as e:
        batch.set_launch("march_rolled")
    assert e.value.status == mdf.MDF_E_INVALID
    assert batch.info()["kernel"] in ("march", "tile")
