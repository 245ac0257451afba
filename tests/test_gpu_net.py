"""GPU parity of the warm-start network (BF16 tensor-core kernels through
include/mdf_net.h: the tcgen05 convolutions with tensor-memory accumulators,
and the mma.sync kernel they replace) against the FP64 network oracle
(oracle/net_oracle.py).

Tolerances: the forward pass is compared with the oracle's BF16-storage mode
(weights, input, every pre-activation, activation and pooled tensor rounded
to BF16 at the points where the GPU stores them; FP64 arithmetic), so the
two differ only by FP32 accumulation order and the rare BF16 rounding flip
that it causes (one BF16 unit, 2^-8 relative, on the affected element).
Gradients are compared with the pure FP64 oracle at the same BF16 weights:
BF16 storage of the activations and of the gradients flowing back (unit
roundoff 2^-9, 15 layers) leaves the GPU gradient within about 1 % of it
(measured 0.4 %), far inside the O(1) error of a wiring or transposition
mistake.
"""
import numpy as np
import pytest

from oracle import net_oracle as N
from paper_2306_08216_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU runs deselect with -m "not gpu"
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2306_08216_gb300 import build as B  # noqa: E402
from paper_2306_08216_gb300 import warmstart  # noqa: E402

B.build()


def case(R, batch, seed):
    p = W.net_init_params(N.layer_shapes(), seed=seed, out_gain=1.0)
    re, n = W.warm_start_draws(batch, seed + 100)
    x = W.warm_start_inputs(re, n, R)
    t = np.random.default_rng(seed + 200).standard_normal((batch, 3, R, R)).astype(np.float32)
    return p, x, t


def test_layer_table_matches_the_oracle():
    net = warmstart.Net(16, 2)
    assert net.layer_shapes() == [(co, ci) for _, co, ci in N.layer_shapes()]
    assert net.param_count == N.param_count()
    p = W.net_init_params(N.layer_shapes(), seed=1)
    net.set_params(p)
    np.testing.assert_array_equal(net.get_params(), p)


@pytest.mark.parametrize("kind", ["tcgen05", "mma.sync"])
@pytest.mark.parametrize("R,batch", [(8, 1), (16, 3), (32, 2)])
def test_forward_matches_bf16_oracle(R, batch, kind):
    p, x, _ = case(R, batch, 7)
    net = warmstart.Net(R, 4)
    net.set_conv_kernel(kind)
    net.set_params(p)
    y = net.forward(x).astype(np.float64)
    ref = N.forward(p, x, quantize=True)
    rel = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    print("forward R=%d rel L2 %.3e max %.3e" % (R, rel, np.abs(y - ref).max() / np.abs(ref).max()))
    assert rel <= 4e-3
    assert np.abs(y - ref).max() <= 2e-2 * np.abs(ref).max()


def test_forward_on_device_buffers():
    R, batch = 16, 2
    p, x, _ = case(R, batch, 8)
    net = warmstart.Net(R, batch)
    net.set_params(p)
    host = net.forward(x)
    dev = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    np.testing.assert_array_equal(host, dev)


@pytest.mark.parametrize("kind", ["tcgen05", "mma.sync"])
def test_gradient_matches_fp64_oracle(kind):
    R, batch = 16, 2
    p, x, t = case(R, batch, 9)
    net = warmstart.Net(R, batch)
    net.set_conv_kernel(kind)
    net.set_params(p)
    loss, g = net.gradient(x, t)
    # the oracle differentiates at the BF16-rounded weights the GPU uses
    pq = torch.tensor(p).to(torch.bfloat16).to(torch.float64).numpy()
    pq[_bias_mask()] = p[_bias_mask()]
    Lo, go = N.loss_and_grad(pq, x, t)
    assert loss == pytest.approx(Lo, rel=2e-2)
    cos = float(g @ go / (np.linalg.norm(g) * np.linalg.norm(go)))
    rel = float(np.linalg.norm(g - go) / np.linalg.norm(go))
    print("gradient cos %.6f rel %.3e" % (cos, rel))
    assert cos >= 0.9995 and rel <= 2e-2
    k = 0
    for name, co, ci in N.layer_shapes():
        n = co * 9 * ci + co
        a, b = g[k:k + n], go[k:k + n]
        lr = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        print("  %s rel %.3e" % (name, lr))
        assert lr <= 3e-2, name
        k += n


def test_tcgen05_forward_at_the_trained_resolution():
    """R = 128, the resolution the shipped network runs at: every layer shape
    (32-256 channels, 128^2 down to 16^2 pixels, every N tile width) on the
    tcgen05 kernel against the mma.sync kernel, which accumulates the same
    K = 16 products in the same order (measured equal to the bit), and
    against the BF16-storage oracle.  Against the oracle the FP32 sums differ
    from the FP64 ones by about 1e-6 relative, which flips the BF16 rounding
    of a few elements per 10^4 at each of the 30 rounding points; each flip
    (2^-8 relative) then spreads through the later layers, so the relative
    L2 difference grows with depth and field size: 2e-3 at R <= 32,
    3.6e-3 at R = 128 in a first measurement; the bound here is 1e-2 (a
    wiring, transposition or layout error is O(1))."""
    R, batch = 128, 2
    p, x, _ = case(R, batch, 11)
    net = warmstart.Net(R, batch)
    net.set_params(p)
    y_tc = net.forward(x).astype(np.float64)
    net.set_conv_kernel("mma.sync")
    y_ms = net.forward(x).astype(np.float64)
    ref = N.forward(p, x, quantize=True)
    rel = np.linalg.norm(y_tc - ref) / np.linalg.norm(ref)
    rel_ms = np.linalg.norm(y_tc - y_ms) / np.linalg.norm(y_ms)
    print("R=128 forward rel L2 vs oracle %.3e (max %.3e), vs mma.sync %.3e"
          % (rel, np.abs(y_tc - ref).max() / np.abs(ref).max(), rel_ms))
    assert rel_ms <= 4e-3
    assert rel <= 1e-2
    assert np.abs(y_tc - ref).max() <= 5e-2 * np.abs(ref).max()


def test_tcgen05_equals_mma_sync_at_the_training_batch():
    """R = 128 with the training batch of 16: enough pixels for the tcgen05
    kernel's tiles of four 128-pixel blocks on the 32-channel layers and
    its widest N tiles elsewhere.  Forward outputs equal to the bit, the
    parameter gradient to the order of its FP32 atomic sums."""
    R, batch = 128, 16
    p, x, t = case(R, batch, 12)
    net = warmstart.Net(R, batch)
    net.set_params(p)
    res = {}
    for kind in ("tcgen05", "mma.sync"):
        net.set_conv_kernel(kind)
        res[kind] = (net.forward(x), net.gradient(x, t))
    np.testing.assert_array_equal(res["tcgen05"][0], res["mma.sync"][0])
    g1, g0 = res["tcgen05"][1][1], res["mma.sync"][1][1]
    rel = float(np.linalg.norm(g1 - g0) / np.linalg.norm(g0))
    print("batch 16 gradient rel diff %.3e" % rel)
    assert rel <= 1e-6


def _bias_mask():
    m = np.zeros(N.param_count(), dtype=bool)
    k = 0
    for _, co, ci in N.layer_shapes():
        k += co * 9 * ci
        m[k:k + co] = True
        k += co
    return m


def test_training_reduces_the_loss():
    R, batch = 16, 4
    p, x, _ = case(R, batch, 10)
    p[-3:] = 0.0
    # a smooth target the network can fit
    X, Y = np.meshgrid(np.linspace(0, 1, R), np.linspace(0, 1, R))
    t = np.stack([np.stack([np.sin(np.pi * X) * np.sin(np.pi * Y) * (1 + 0.5 * x[b, 0, 0, 0]),
                            np.cos(np.pi * X) * Y, X * Y * x[b, 1, 0, 0]]) for b in range(batch)]).astype(np.float32)
    net = warmstart.Net(R, batch)
    net.set_params(p)
    first = net.train_step(x, t, 1e-3)
    for _ in range(150):
        last = net.train_step(x, t, 1e-3)
    print("loss %.4e -> %.4e" % (first, last))
    assert last < 0.1 * first
    # the parameters moved and stay finite
    q = net.get_params()
    assert np.isfinite(q).all() and np.abs(q - p).max() > 0


def test_invalid_arguments():
    from paper_2306_08216_gb300 import mdf
    with pytest.raises(mdf.MdfError):
        warmstart.Net(12, 1)  # not a multiple of 8
    net = warmstart.Net(8, 2)
    with pytest.raises(AssertionError):
        net.set_params(np.zeros(5, dtype=np.float32))
    x = np.zeros((3, 8, 8, 8), dtype=np.float32)
    with pytest.raises(mdf.MdfError):
        net.forward(x)  # batch above max_batch
