"""What the trained warm-start network gains: held-out power-law cavities
(seeded draws the network never saw) marched to a residual target from rest
and from the network's prediction, with the shipped parameters
(paper_2306_08216_gb300/weights/warmstart_cavity_R128.npy)."""
import os

import numpy as np
import pytest

from paper_2306_08216_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2306_08216_gb300 import build as B  # noqa: E402
from paper_2306_08216_gb300 import mdf  # noqa: E402
from paper_2306_08216_gb300 import warmstart as WS  # noqa: E402

B.build()

R = 128
WEIGHTS = os.path.join(WS.WEIGHTS_DIR, "warmstart_cavity_R128.npy")
HOLDOUT_SEED, HOLDOUT_COUNT = 2, 64  # the training set is seed 1 (1024 draws)


@pytest.fixture(scope="module")
def net():
    n = WS.Net(R, 8)
    n.load(WEIGHTS)
    return n


@pytest.fixture(scope="module")
def holdout():
    re, nn = W.warm_start_draws(HOLDOUT_COUNT, HOLDOUT_SEED)
    return re[:8], nn[:8]


def test_prediction_error_on_held_out_cavities(net, holdout):
    """Steady states from the solver (residual 1e-6) against the network's
    predictions: a few percent at most in velocity."""
    re, nn = holdout
    batch = mdf.Batch([WS.cavity_problem(R, a, b) for a, b in zip(re, nn)])
    conv, r, st, steps, _ = WS.march(batch, 1e-6, max_steps=150_000)
    assert (st != mdf.MDF_E_DIVERGED).all()
    t = WS.steady_fields(batch)
    eu, ep = WS.evaluate(net, W.warm_start_inputs(re, nn, R), t)
    print("held-out velocity error median %.4f max %.4f, pressure median %.4f" % (np.median(eu), eu.max(),
                                                                                 np.median(ep)))
    assert np.median(eu) < 0.02 and eu.max() < 0.05


def test_warm_start_reaches_the_target_in_fewer_steps(net, holdout):
    re, nn = holdout
    out = WS.warm_vs_cold(net, re, nn, R, target=1e-6, max_steps=120_000, log=None)
    print({k: v for k, v in out.items() if k not in ("cold", "warm")})
    assert out["reached_both"] >= 4
    assert out["median_step_ratio_cold_over_warm"] >= 3.0
    assert out["speedup_warm_batch_vs_cold_batch"] > 1.5


def test_warm_and_cold_starts_reach_the_same_steady_state(net, holdout):
    """The network only moves the starting point: marched to residual 1e-8,
    the warm and cold runs of a cavity that converges agree to the distance
    from steady state that this residual leaves.  This cavity's residual
    falls two decades in about 33,000 steps near the end (a factor 0.87 per
    1000-step window), so a windowed residual of 1e-8 (relative change 1e-5
    per window) leaves each run about 1e-5 / 0.13 = 8e-5 (relative L2) from
    the steady state; the max-norm gap is larger, concentrated at the lid
    corners."""
    re, nn = holdout
    k = 1  # Re 199, n 1.33: converges below 1e-8 from both starts
    probs = [WS.cavity_problem(R, re[k], nn[k])]
    y = net.forward(W.warm_start_inputs(re[k:k + 1], nn[k:k + 1], R))
    states = []
    for warm in (False, True):
        b = mdf.Batch(probs)
        if warm:
            b.init(0, y[0, 0] * WS.U_LID, y[0, 1] * WS.U_LID, y[0, 2] * WS.U_LID ** 2)
        conv, r, st, steps, _ = WS.march(b, 1e-8, max_steps=200_000)
        assert conv[0] > 0, r
        states.append(b.problem(0).fields(["u", "v"]))
    du = max(float(np.abs(states[0][c] - states[1][c]).max()) for c in ("u", "v"))
    num = sum(float(((states[0][c].astype(np.float64) - states[1][c]) ** 2).sum()) for c in ("u", "v"))
    den = sum(float((states[0][c].astype(np.float64) ** 2).sum()) for c in ("u", "v"))
    rel = (num / den) ** 0.5
    print("warm vs cold at 1e-8: relative L2 %.3e, max %.3e u_lid" % (rel, du / WS.U_LID))
    assert rel < 4e-4 and du < 5e-3 * WS.U_LID
