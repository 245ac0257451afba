"""Lid-driven cavity on the GPU against the paper's own vortex table.

Sec. 4.4: u0 = 0.1, L = 1, c = 1, CFL 0.5, NEE walls; Re = 400 on a 128 x 128
grid and Re = 1000 on a 256 x 256 grid (walls on nodes).  The primary-vortex
centre of the steady state (residual 1e-8) must lie within one grid spacing of
the MDF-FDLBM row of the paper's vortex table
(tests/golden/table10_cavity_vortex_centres.json), the two bottom corner
vortices at Re = 1000 within two.
"""
import json
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

B.build()
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table10_cavity_vortex_centres.json")


def vortex_centre(u, x, y):
    """Minimum of the stream function psi = int_0^y u dy, refined by a
    three-point parabola in each direction."""
    psi = np.zeros_like(u)
    psi[1:] = np.cumsum(0.5 * (u[1:] + u[:-1]) * np.diff(y)[:, None], axis=0)
    j, i = np.unravel_index(np.argmin(psi), psi.shape)

    def refine(v, k, c):
        a, b, d = v[k - 1], v[k], v[k + 1]
        den = a - 2 * b + d
        return c[k] + (0.5 * (a - d) / den if den else 0.0) * (c[k + 1] - c[k - 1]) / 2

    return refine(psi[j, :], i, x), refine(psi[:, i], j, y)


def test_cavity_re400_primary_vortex_matches_paper():
    table = json.load(open(GOLDEN))
    ref = table["primary"][table["Re"].index(400)]
    n, u0, Re = 129, 0.1, 400.0
    s = mdf.Solver(n, n, nu=u0 / Re, walls=(True, True), u_wall=(0, 0, 0, u0))
    s.init(*W.zeros(n, n))
    r, steps = 1.0, 0
    while r > 1e-8 and steps < 400_000:
        s.step(100)
        steps += 100
        r, _ = s.residual()
    assert r <= 1e-8, (r, steps)
    x = W.wall_nodes(n, 1.0)
    xc, yc = vortex_centre(s.fields(["u"])["u"].astype(np.float64), x, x)
    h = 1.0 / (n - 1)
    assert abs(xc - ref[0]) <= h and abs(yc - ref[1]) <= h, ((xc, yc), ref)


def corner_vortex_centre(u, x, y, xr, yr):
    """Maximum of psi (the counter-rotating corner vortex) inside the box
    xr x yr, refined by a three-point parabola in each direction."""
    psi = np.zeros_like(u)
    psi[1:] = np.cumsum(0.5 * (u[1:] + u[:-1]) * np.diff(y)[:, None], axis=0)
    mi = (x >= xr[0]) & (x <= xr[1])
    mj = (y >= yr[0]) & (y <= yr[1])
    sub = np.where(mj[:, None] & mi[None, :], psi, -np.inf)
    j, i = np.unravel_index(np.argmax(sub), sub.shape)

    def refine(v, k, c):
        a, b, d = v[k - 1], v[k], v[k + 1]
        den = a - 2 * b + d
        return c[k] + (0.5 * (a - d) / den if den else 0.0) * (c[k + 1] - c[k - 1]) / 2

    return refine(psi[j, :], i, x), refine(psi[:, i], j, y)


def test_cavity_re1000_vortices_match_paper():
    """Re = 1000 on the paper's 256 x 256 grid (257 nodes per side), marched
    from rest to residual 1e-8: the primary vortex within one grid spacing of
    the paper's MDF-FDLBM centre, the two bottom corner vortices within two."""
    table = json.load(open(GOLDEN))
    k = table["Re"].index(1000)
    n, u0, Re = 257, 0.1, 1000.0
    s = mdf.Solver(n, n, nu=u0 / Re, walls=(True, True), u_wall=(0, 0, 0, u0))
    s.init(*W.zeros(n, n))
    r, steps = 1.0, 0
    while r > 1e-8 and steps < 800_000:
        s.step(100)
        steps += 100
        r, _ = s.residual()
    assert r <= 1e-8, (r, steps)
    x = W.wall_nodes(n, 1.0)
    u = s.fields(["u"])["u"].astype(np.float64)
    h = 1.0 / (n - 1)
    xc, yc = vortex_centre(u, x, x)
    ref = table["primary"][k]
    assert abs(xc - ref[0]) <= h and abs(yc - ref[1]) <= h, ((xc, yc), ref)
    for key, box in (("bottom_left", ((0.0, 0.3), (0.0, 0.3))), ("bottom_right", ((0.6, 1.0), (0.0, 0.4)))):
        ref = table[key][k]
        xs, ys = corner_vortex_centre(u, x, x, *box)
        assert abs(xs - ref[0]) <= 2 * h and abs(ys - ref[1]) <= 2 * h, (key, (xs, ys), ref)
