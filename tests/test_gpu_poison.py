"""Out-of-stencil reads, caught without a memory checker: NaN is written into
every storage element no valid result may read (row padding, and the ghost
columns beside x walls; mdf_debug_poison), and the poisoned run must equal the
clean one bit for bit.  Every kernel family, storage mode and wall layout, on
ragged grids, with graph replay and single launches."""
import numpy as np
import pytest

from paper_2306_08216_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2306_08216_gb300 import build as B  # noqa: E402
from paper_2306_08216_gb300 import mdf  # noqa: E402

B.build()

LID = dict(walls=(True, True), u_wall=(0, 0, 0, 0.1))
PL = dict(power_law=(0.004, 0.8, 2e-4, 0.08))
TRAP = W.trapezoid_grid(37, 37)
STRETCH = 0.5 * (1 + np.tanh(1.5 * (2 * np.arange(41) / 40 - 1)) / np.tanh(1.5))

CASES = {
    # name: (nx, ny, solver keywords, plans: (threads, rows) or (0, 0) for the tile kernel)
    "periodic": (45, 37, dict(nu=0.01, lx=1.0, ly=37 / 45), [(256, 6), (128, 4), (0, 0)]),
    "periodic_fp16": (45, 37, dict(nu=0.01, lx=1.0, ly=37 / 45, storage="fp16"), [(256, 6), (0, 0)]),
    "periodic_bf16_forced": (45, 37, dict(nu=0.01, lx=1.0, ly=37 / 45, storage="bf16", force=(1e-4, 0.0)),
                             [(128, 4), (0, 0)]),
    "cavity": (45, 37, dict(nu=0.01, **LID), [(128, 3), (256, 8), (0, 0)]),
    "channel": (45, 37, dict(nu=0.01, lx=1.0, walls=(False, True), force=(1e-4, 0.0)), [(128, 3), (0, 0)]),
    "x_walls": (45, 37, dict(nu=0.01, ly=1.0, walls=(True, False), u_wall=(0, 0, 0, 0), v_wall=(0.05, -0.05, 0, 0)),
                [(128, 5), (0, 0)]),
    "power_law_cavity": (45, 37, dict(nu=0.004, **LID, **PL), [(128, 2), (0, 0)]),
    "power_law_fp16": (45, 37, dict(nu=0.004, storage="fp16", **LID, **PL), [(0, 0)]),
    "stretched_cavity": (41, 41, dict(nu=0.01, grid="separable", x=STRETCH, y=STRETCH, **LID), [(128, 4), (0, 0)]),
    "trapezoid": (37, 37, dict(nu=0.01, grid="curvilinear", x=TRAP[0], y=TRAP[1], **LID), [(128, 3), (0, 0)]),
    "trapezoid_power_law": (37, 37, dict(nu=0.004, grid="curvilinear", x=TRAP[0], y=TRAP[1], **LID, **PL),
                            [(128, 3), (0, 0)]),
    "rho0_cavity": (45, 37, dict(nu=0.01, rho0=True, **LID), [(128, 3), (0, 0)]),
}


def run(nx, ny, kw, plan, poison, steps=70):
    s = mdf.Solver(nx, ny, **kw)
    s.set_launch(*plan)
    u, v, p = W.random_fields(nx, ny, 0.02, 5)
    s.init(u, v, p)
    if poison:
        s.debug_poison()
    s.step(steps - 5)   # graph replays and single launches
    for _ in range(5):
        s.step(1)
    out = [s.state()]
    if kw.get("rho0"):
        out.append(s.rho0_state())
    return out


@pytest.mark.parametrize("name", sorted(CASES))
def test_poisoned_storage_is_never_read(name):
    nx, ny, kw, plans = CASES[name]
    for plan in plans:
        clean, dirty = run(nx, ny, kw, plan, False), run(nx, ny, kw, plan, True)
        for a, b in zip(clean, dirty):
            assert np.isfinite(b).all(), (name, plan)
            np.testing.assert_array_equal(a, b, err_msg="%s %s" % (name, plan))


@pytest.mark.parametrize("kernel", ["march", "march_rolled", "tile"])
def test_poisoned_batch(kernel):
    probs = [dict(nx=n, ny=n, nu=0.004, **LID, **PL) for n in (45, 33, 70)]
    states = []
    for poison in (False, True):
        b = mdf.Batch(probs)
        b.set_launch(kernel)
        if poison:
            for i in range(len(probs)):
                b.problem(i).debug_poison()
        b.step(40)
        b.step(3)
        states.append([b.problem(i).state() for i in range(len(probs))])
    for a, c in zip(*states):
        np.testing.assert_array_equal(a, c)
