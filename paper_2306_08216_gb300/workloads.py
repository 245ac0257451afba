"""Seeded synthetic workloads (initial fields, body forces, grids).

This module only generates inputs: analytic initial/forcing fields of the
paper's test problems and node coordinates of the grids.  It holds none of the
method's arithmetic and imports neither the CUDA binding nor the oracle, so
both sides can be fed the same inputs.

Problems (arXiv:2306.08216 Sec. 4 unless noted):
  taylor_green   decaying Taylor-Green vortex on [0, 2pi]^2 (textbook closed form)
  four_roll_mill Sec. 4.1, Eqs. 4.1.1-4.1.2, periodic [0, 2pi]^2
  periodic_flow  Sec. 4.2, Eqs. 4.2.1-4.2.2, periodic [0, 1]^2
  poiseuille     Sec. 4.3, Eq. 4.3.1, channel [0,1]^2, walls at y = 0, 1
  cavity         Sec. 4.4, lid-driven square cavity, lid speed u0
Grids: uniform, tanh-stretched (separable) and a trapezoid mapped from the
unit square (curvilinear).

Warm-start network inputs (the network is the project's extension, not the
paper's): seeded initial parameters, the eight input planes of a cavity
(Re, power-law index, node coordinates, metric coefficients) and seeded
(Re, n) draws.
"""
import math

import numpy as np


def periodic_nodes(n, length):
    """Nodes x_i = i * length / n of a periodic axis."""
    return np.arange(n, dtype=np.float64) * (length / n)


def wall_nodes(n, length):
    """Nodes x_i = i * length / (n - 1), walls on the first and last node."""
    return np.arange(n, dtype=np.float64) * (length / (n - 1))


def tanh_nodes(n, beta, length=1.0):
    """Wall-clustered nodes x_i = L/2 [1 + tanh(beta (2 i/(n-1) - 1)) / tanh(beta)]."""
    s = np.arange(n, dtype=np.float64) / (n - 1)
    return 0.5 * length * (1.0 + np.tanh(beta * (2.0 * s - 1.0)) / math.tanh(beta))


def trapezoid_grid(nx, ny, bottom=0.5, top=1.0, height=1.0):
    """Isosceles trapezoid (bottom width `bottom`, lid width `top`, height
    `height`), mapped from the unit square by linear blending between the two
    slanted side walls.  Returns X, Y of shape (ny, nx)."""
    xi = np.arange(nx, dtype=np.float64) / (nx - 1)
    et = np.arange(ny, dtype=np.float64) / (ny - 1)
    XI, ET = np.meshgrid(xi, et)
    half = 0.5 * (bottom + (top - bottom) * ET)
    X = 0.5 * top - half + 2.0 * half * XI
    Y = height * ET
    return X, Y


def trapezoid_metrics(nx, ny, bottom=0.5, top=1.0, height=1.0):
    """Exact metric coefficients of trapezoid_grid per unit node index:
    x_i = 2 half/(nx - 1), x_j = (top - bottom)(xi - 1/2)/(ny - 1), y_i = 0,
    y_j = height/(ny - 1), inverted.  Returns xi_x, xi_y, eta_x, eta_y."""
    xi = np.arange(nx, dtype=np.float64) / (nx - 1)
    et = np.arange(ny, dtype=np.float64) / (ny - 1)
    XI, ET = np.meshgrid(xi, et)
    half = 0.5 * (bottom + (top - bottom) * ET)
    x_i = 2.0 * half / (nx - 1)
    x_j = (top - bottom) * (XI - 0.5) / (ny - 1)
    y_j = np.full_like(XI, height / (ny - 1))
    J = x_i * y_j
    return y_j / J, -x_j / J, np.zeros_like(XI), x_i / J


def taylor_green(n, U0=0.01, length=2.0 * math.pi):
    """u = -U0 cos x sin y, v = U0 sin x cos y, p = -(U0^2/4)(cos 2x + cos 2y)
    on the periodic square [0, L)^2 with L = 2 pi (k = 2 pi / L)."""
    x = periodic_nodes(n, length)
    k = 2.0 * math.pi / length
    X, Y = np.meshgrid(x, x)
    u = -U0 * np.cos(k * X) * np.sin(k * Y)
    v = U0 * np.sin(k * X) * np.cos(k * Y)
    p = -(U0 * U0 / 4.0) * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    return u, v, p


def taylor_green_exact(n, t, nu, U0=0.01, length=2.0 * math.pi):
    """Closed form at time t: the fields above times exp(-2 nu k^2 t) (p: squared)."""
    u, v, p = taylor_green(n, U0, length)
    k = 2.0 * math.pi / length
    d = math.exp(-2.0 * nu * k * k * t)
    return u * d, v * d, p * d * d


def four_roll_mill(n, U0=1e-4, nu=0.01):
    """Eqs. 4.1.1-4.1.2 on [0, 2pi)^2.  The force on the second component uses
    the sign that makes the printed velocity a steady solution with P = 0:
    F2 = U0^2 sin y cos y - 2 nu U0 sin y cos x."""
    x = periodic_nodes(n, 2.0 * math.pi)
    X, Y = np.meshgrid(x, x)
    u = U0 * np.sin(X) * np.cos(Y)
    v = -U0 * np.sin(Y) * np.cos(X)
    Fx = U0 * U0 * np.sin(X) * np.cos(X) + 2.0 * nu * U0 * np.sin(X) * np.cos(Y)
    Fy = U0 * U0 * np.sin(Y) * np.cos(Y) - 2.0 * nu * U0 * np.sin(Y) * np.cos(X)
    grads = {
        "dudx": U0 * np.cos(X) * np.cos(Y), "dudy": -U0 * np.sin(X) * np.sin(Y),
        "dvdx": U0 * np.sin(X) * np.sin(Y), "dvdy": -U0 * np.cos(X) * np.cos(Y),
    }
    return u, v, np.zeros_like(u), Fx, Fy, grads


def distorted_periodic_grid(n, a):
    """Doubly periodic non-affine grid of n x n nodes on [0, 1)^2:
    x = xi + a sin(2 pi eta), y = eta + a sin(2 pi xi), xi, eta = i/n
    (a < 1/(2 pi) keeps the map one-to-one).  Returns X, Y [n, n]."""
    xi = np.arange(n) / n
    XI, ETA = np.meshgrid(xi, xi)
    return XI + a * np.sin(2 * math.pi * ETA), ETA + a * np.sin(2 * math.pi * XI)


def distorted_periodic_metrics(n, a):
    """Exact metric coefficients of distorted_periodic_grid(n, a) per unit
    node index (the computational coordinates step by one per node):
    xi_x, xi_y, eta_x, eta_y [n, n] from the derivatives of the mapping,
    x_i = 1/n, x_j = (2 pi a/n) cos(2 pi eta), y_i = (2 pi a/n) cos(2 pi xi),
    y_j = 1/n, and the inverse of the Jacobian matrix."""
    xi = np.arange(n) / n
    XI, ETA = np.meshgrid(xi, xi)
    x_i = np.full((n, n), 1.0 / n)
    x_j = (2 * math.pi * a / n) * np.cos(2 * math.pi * ETA)
    y_i = (2 * math.pi * a / n) * np.cos(2 * math.pi * XI)
    y_j = np.full((n, n), 1.0 / n)
    J = x_i * y_j - x_j * y_i
    return y_j / J, -x_j / J, -y_i / J, x_i / J


def periodic_flow_at(X, Y, u0=0.1, nu=0.01):
    """Eqs. 4.2.1-4.2.2 sampled at arbitrary node coordinates: u, v, Fx, Fy."""
    tp = 2.0 * math.pi
    u = u0 * np.sin(tp * X) * np.sin(tp * Y)
    v = u0 * np.cos(tp * X) * np.cos(tp * Y)
    return u, v, 8.0 * math.pi ** 2 * nu * u, 8.0 * math.pi ** 2 * nu * v


def periodic_flow(nx, ny, u0=0.1, nu=0.01, rho0=1.0):
    """Eqs. 4.2.1-4.2.2 on [0, 1)^2 (nx x ny nodes): steady u, v, p and the force."""
    X, Y = np.meshgrid(periodic_nodes(nx, 1.0), periodic_nodes(ny, 1.0))
    tp = 2.0 * math.pi
    u = u0 * np.sin(tp * X) * np.sin(tp * Y)
    v = u0 * np.cos(tp * X) * np.cos(tp * Y)
    p = 0.25 * rho0 * u0 * u0 * (np.cos(2 * tp * X) - np.cos(2 * tp * Y))
    Fx = 8.0 * math.pi ** 2 * nu * u0 * np.sin(tp * X) * np.sin(tp * Y)
    Fy = 8.0 * math.pi ** 2 * nu * u0 * np.cos(tp * X) * np.cos(tp * Y)
    grads = {
        "dudx": tp * u0 * np.cos(tp * X) * np.sin(tp * Y),
        "dudy": tp * u0 * np.sin(tp * X) * np.cos(tp * Y),
        "dvdx": -tp * u0 * np.sin(tp * X) * np.cos(tp * Y),
        "dvdy": -tp * u0 * np.cos(tp * X) * np.sin(tp * Y),
    }
    return u, v, p, Fx, Fy, grads


def poiseuille_exact(y, F, nu, H=1.0):
    """Eq. 4.3.1: u = F H^2/(2 nu) [y/H - (y/H)^2] and du/dy."""
    u = F * H * H / (2.0 * nu) * (y / H - (y / H) ** 2)
    dudy = F * H / (2.0 * nu) * (1.0 - 2.0 * y / H)
    return u, dudy


def power_law_poiseuille_exact(y, G, K, n, H=1.0):
    """Fully developed channel flow of a power-law fluid, nu = K gdot^(n-1):
    u = n/(n+1) (G/K)^(1/n) [(H/2)^(1+1/n) - |y - H/2|^(1+1/n)]."""
    e = 1.0 + 1.0 / n
    return n / (n + 1.0) * (G / K) ** (1.0 / n) * ((H / 2.0) ** e - np.abs(y - H / 2.0) ** e)


def zeros(nx, ny):
    z = np.zeros((ny, nx), dtype=np.float64)
    return z, z.copy(), z.copy()


def random_state(nx, ny, amplitude, seed):
    """Seeded random distributions fhat[alpha, j, y, x] (normal, std = amplitude)."""
    rng = np.random.default_rng(seed)
    return amplitude * rng.standard_normal((2, 5, ny, nx))


def random_fields(nx, ny, amplitude, seed):
    """Seeded smooth-ish random u, v, p fields (sum of a few low Fourier modes)."""
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(np.arange(nx) / nx, np.arange(ny) / ny)
    out = []
    for _ in range(3):
        f = np.zeros((ny, nx))
        for _ in range(4):
            kx, ky = rng.integers(1, 4, size=2)
            ph = rng.uniform(0, 2 * math.pi, size=2)
            f += rng.standard_normal() * np.sin(2 * math.pi * kx * X + ph[0]) * np.cos(2 * math.pi * ky * Y + ph[1])
        out.append(amplitude * f)
    return out


def cavity_batch_draws(count, seed=2306):
    """Seeded draws for a sweep of cavities: Re log-uniform in [100, 5000],
    power-law index uniform in [0.5, 1.5], grid side in {65, 129, 257, 513}."""
    rng = np.random.default_rng(seed)
    re = np.exp(rng.uniform(math.log(100.0), math.log(5000.0), size=count))
    n = rng.uniform(0.5, 1.5, size=count)
    sides = rng.choice(np.array([65, 129, 257, 513]), size=count)
    return re, n, sides


# ---------------------------------------------------------------- warm start

WARM_RE_RANGE = (100.0, 1000.0)
WARM_N_RANGE = (0.5, 1.5)


def warm_start_draws(count, seed):
    """Seeded power-law cavity parameters: Re log-uniform in [100, 1000],
    index n uniform in [0.5, 1.5]."""
    rng = np.random.default_rng(seed)
    re = np.exp(rng.uniform(math.log(WARM_RE_RANGE[0]), math.log(WARM_RE_RANGE[1]), size=count))
    n = rng.uniform(WARM_N_RANGE[0], WARM_N_RANGE[1], size=count)
    return re, n


WARM_IN_PLANES = 8


def warm_start_inputs(re, n_index, R, geometry="square"):
    """Input planes [B][8][R][R] (float32) of the warm-start network: the
    scaled log Reynolds number and power-law index (each mapped to [-1, 1]
    over the training ranges), the node coordinates x, y of the cavity grid
    and its four metric coefficients xi_x, xi_y, eta_x, eta_y, the
    derivatives of the computational coordinates xi = i/(R-1), eta = j/(R-1)
    with respect to x and y.  geometry "square": the unit square (x = xi,
    y = eta, metrics 1, 0, 0, 1); "trapezoid": trapezoid_grid(R, R) and its
    exact metrics; or a sequence of those names, one per sample."""
    re = np.atleast_1d(np.asarray(re, dtype=np.float64))
    n_index = np.atleast_1d(np.asarray(n_index, dtype=np.float64))
    geo = [geometry] * re.size if isinstance(geometry, str) else list(geometry)
    assert len(geo) == re.size
    lo, hi = math.log(WARM_RE_RANGE[0]), math.log(WARM_RE_RANGE[1])
    a = 2.0 * (np.log(re) - lo) / (hi - lo) - 1.0
    b = 2.0 * (n_index - WARM_N_RANGE[0]) / (WARM_N_RANGE[1] - WARM_N_RANGE[0]) - 1.0
    planes = {}
    X, Y = np.meshgrid(np.arange(R) / (R - 1.0), np.arange(R) / (R - 1.0))
    one, zero = np.ones_like(X), np.zeros_like(X)
    planes["square"] = (X, Y, one, zero, zero, one)
    if "trapezoid" in geo:
        Xt, Yt = trapezoid_grid(R, R)
        m = trapezoid_metrics(R, R)  # d(index)/dx: divide by R - 1 for d(xi)/dx
        planes["trapezoid"] = (Xt, Yt) + tuple(c / (R - 1.0) for c in m)
    out = np.empty((re.size, WARM_IN_PLANES, R, R), dtype=np.float32)
    for k in range(re.size):
        out[k, 0] = a[k]
        out[k, 1] = b[k]
        for c, plane in enumerate(planes[geo[k]]):
            out[k, 2 + c] = plane
    return out


def net_init_params(shapes, seed, out_gain=0.1):
    """Seeded initial parameters of a stack of 3 x 3 convolutions, flat
    float32 in the order of `shapes` = [(name, cout, cin), ...]: weights
    [cout][3][3][cin] normal with std sqrt(2 / (9 cin)) (He), scaled by
    out_gain on the last layer, then zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, (_, co, ci) in enumerate(shapes):
        std = math.sqrt(2.0 / (9.0 * ci)) * (out_gain if i == len(shapes) - 1 else 1.0)
        parts.append((std * rng.standard_normal(co * 9 * ci)).astype(np.float32))
        parts.append(np.zeros(co, dtype=np.float32))
    return np.concatenate(parts)
