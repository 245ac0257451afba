"""Pins of the warm-start network oracle (oracle/net_oracle.py) against
facts that do not come from the oracle itself: brute-force convolution on
tiny inputs, closed forms of pooling / upsampling and of the skip wiring, and
finite-difference derivatives of the loss."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import net_oracle as N  # noqa: E402
from paper_2306_08216_gb300 import workloads as W  # noqa: E402


def silu(z):
    return z / (1.0 + math.exp(-z))


def test_conv3x3_matches_brute_force_sum():
    rng = np.random.default_rng(1)
    B, ci, co, R = 2, 3, 2, 5
    h = rng.standard_normal((B, ci, R, R))
    w = rng.standard_normal((co, 3, 3, ci))
    b = rng.standard_normal(co)
    got = N.conv3x3(torch.tensor(h), torch.tensor(w), torch.tensor(b)).numpy()
    ref = np.zeros((B, co, R, R))
    for n in range(B):
        for o in range(co):
            for y in range(R):
                for x in range(R):
                    acc = b[o]
                    for i in range(3):
                        for j in range(3):
                            yy, xx = y + i - 1, x + j - 1
                            if 0 <= yy < R and 0 <= xx < R:
                                acc += sum(w[o, i, j, c] * h[n, c, yy, xx] for c in range(ci))
                    ref[n, o, y, x] = acc
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


def test_parameter_count_and_shapes():
    shapes = N.layer_shapes()
    assert [s[0] for s in shapes][0] == "e0a" and shapes[-1] == ("out", 3, 32)
    assert N.param_count() == sum(co * 9 * ci + co for _, co, ci in shapes)
    assert 1.5e6 < N.param_count() < 2.5e6  # a ~2M-parameter network


def _blank():
    return np.zeros(N.param_count())


def _offsets():
    off, k = {}, 0
    for name, co, ci in N.layer_shapes():
        off[name] = (k, co, ci)
        k += co * 9 * ci + co
    return off


def _set_identity(p, name, off):
    """Centre tap = identity between the first min(cin, cout) channels."""
    k, co, ci = off[name]
    w = p[k:k + co * 9 * ci].reshape(co, 3, 3, ci)
    for c in range(min(co, ci)):
        w[c, 1, 1, c] = 1.0


def _set_bias(p, name, off, value):
    k, co, ci = off[name]
    p[k + co * 9 * ci:k + co * 9 * ci + co] = value


def test_zero_network_outputs_the_output_bias():
    off = _offsets()
    p = _blank()
    _set_bias(p, "out", off, np.array([0.25, -0.5, 2.0]))
    x = W.warm_start_inputs([300.0], [0.8], 16)
    y = N.forward(p, x)
    for c, v in enumerate([0.25, -0.5, 2.0]):
        assert np.all(y[0, c] == v)


@pytest.mark.parametrize("level", [0, 1, 2])
def test_skip_connection_wiring(level):
    """All weights zero except identity centre taps along the decoder from
    level k down: the encoder output s_k (a constant silu(beta)) enters the
    pre-activation of d_ka, and the output is a closed-form chain of SiLUs."""
    off = _offsets()
    p = _blank()
    beta = 0.7
    _set_bias(p, "e%db" % level, off, beta)          # s_k = silu(beta), constant
    chain = ["d%da" % level, "d%db" % level]
    for k in range(level - 1, -1, -1):
        chain += ["d%da" % k, "d%db" % k]
    for name in chain:
        _set_identity(p, name, off)
    _set_identity(p, "out", off)
    x = W.warm_start_inputs([300.0], [0.8], 16)
    y = N.forward(p, x)
    # d_ka: silu(0 + s_k); every later layer is silu(identity) (the skips of
    # lower levels are silu(silu(0)) = 0 since their biases are zero)
    v = silu(silu(beta))
    for _ in range(len(chain) - 1):
        v = silu(v)
    # every channel carries the same constant through the identity taps
    np.testing.assert_allclose(y[0], v, rtol=1e-14)


def test_pool_and_upsample_closed_forms():
    a = torch.arange(16, dtype=torch.float64).reshape(1, 1, 4, 4)
    pooled = torch.nn.functional.avg_pool2d(a, 2)
    np.testing.assert_array_equal(pooled.numpy()[0, 0], [[2.5, 4.5], [10.5, 12.5]])
    up = torch.nn.functional.interpolate(pooled, scale_factor=2, mode="nearest").numpy()[0, 0]
    np.testing.assert_array_equal(up[:2, :2], 2.5)
    np.testing.assert_array_equal(up[2:, 2:], 12.5)


def test_gradient_matches_finite_differences():
    R, B = 8, 2
    p = W.net_init_params(N.layer_shapes(), seed=3, out_gain=1.0).astype(np.float64)
    rng = np.random.default_rng(4)
    p[-3:] = rng.standard_normal(3)
    x = W.warm_start_inputs([150.0, 700.0], [0.6, 1.3], R)
    t = rng.standard_normal((B, 3, R, R))
    L, g = N.loss_and_grad(p, x, t)
    assert L == pytest.approx(N.loss(p, x, t), rel=1e-14)
    for trial in range(4):
        d = rng.standard_normal(p.size)
        eps = 1e-6
        fd = (N.loss(p + eps * d, x, t) - N.loss(p - eps * d, x, t)) / (2 * eps)
        assert fd == pytest.approx(float(g @ d), rel=1e-6)


def test_quantized_forward_is_close_to_fp64():
    R = 16
    p = W.net_init_params(N.layer_shapes(), seed=5, out_gain=1.0)
    x = W.warm_start_inputs([200.0], [1.1], R)
    a, b = N.forward(p, x), N.forward(p, x, quantize=True)
    rel = np.linalg.norm(a - b) / np.linalg.norm(a)
    assert 0 < rel < 0.05  # BF16 storage of ~15 layers: percent level


def test_input_planes_of_the_two_geometries():
    """The eight input planes: the metric coefficients are derivatives of the
    normalised computational coordinates (1, 0, 0, 1 on the unit square), so
    both geometries give O(1) inputs; on the trapezoid (bottom 0.5, lid 1)
    xi_x = 1 / width runs from 2 at the bottom to 1 at the lid, eta_x = 0,
    eta_y = 1, and xi_y is odd about the centre line."""
    R = 16
    x = W.warm_start_inputs([300.0, 300.0], [0.8, 0.8], R, geometry=["square", "trapezoid"])
    assert x.shape == (2, N.IN_PLANES, R, R)
    sq, tr = x[0], x[1]
    np.testing.assert_array_equal(sq[4:], np.stack([np.ones((R, R)), np.zeros((R, R)), np.zeros((R, R)),
                                                    np.ones((R, R))]).astype(np.float32))
    np.testing.assert_allclose(tr[4][0], 2.0, rtol=1e-6)
    np.testing.assert_allclose(tr[4][-1], 1.0, rtol=1e-6)
    np.testing.assert_allclose(tr[6], 0.0, atol=1e-7)
    np.testing.assert_allclose(tr[7], 1.0, rtol=1e-6)
    np.testing.assert_allclose(tr[5], -tr[5][:, ::-1], atol=1e-6)
    np.testing.assert_allclose(tr[3][:, 0], np.arange(R) / (R - 1.0), rtol=1e-6)
