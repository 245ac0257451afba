"""FP64 CPU oracle of the warm-start network (plain PyTorch CPU ops).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` and never by the library.
It shares no code with the CUDA path (``csrc/net_*.cu``); both are written
from the network specification below.  The paper has no learned component:
this network is the project's warm-start extension, which predicts a steady
lid-driven cavity state so that the MDF-FDLBM march (Sec. 2.2) starts closer
to it.  The method's arithmetic stays in the solver.

Specification (both sides implement exactly this):

* Input: B x 8 x R x R planes (R divisible by 8): scaled log Re, scaled
  power-law index, the node coordinates x, y and the four metric
  coefficients xi_x, xi_y, eta_x, eta_y of the cavity's grid (derivatives of
  the computational coordinates, scaled to [0, 1] over the grid, with respect
  to x and y); output B x 3 x R x R (u / u_lid, v / u_lid, p / u_lid^2 of the
  steady state on the R x R nodes).
* Layers, 3 x 3 convolutions (cross-correlation, zero padding 1, stride 1,
  with bias), in this order:
      e0a 8->32, e0b 32->32          (resolution R)
      e1a 32->64, e1b 64->64         (R/2)
      e2a 64->128, e2b 128->128      (R/4)
      e3a 128->256, e3b 256->256     (R/8)
      d2a 256->128, d2b 128->128     (R/4)
      d1a 128->64, d1b 64->64        (R/2)
      d0a 64->32, d0b 32->32         (R)
      out 32->3                      (R)
  Activation SiLU(z) = z / (1 + exp(-z)) after every layer except `out`.
  Encoder: x -> e0a -> e0b = s0 -> pool -> e1a -> e1b = s1 -> pool -> e2a
  -> e2b = s2 -> pool -> e3a -> e3b.  Decoder level k: up -> dka, whose
  pre-activation is conv + bias + s_k, -> dkb.  pool = 2 x 2 average,
  up = nearest-neighbour x 2.
* Parameters: one flat float vector, layer by layer: weights [Cout][3][3][Cin]
  (kernel row i, column j: input offset (i - 1, j - 1) in (y, x)), then
  bias [Cout].
* Loss: mean over B x 3 x R x R of (out - target)^2.

``quantize=True`` rounds what the GPU stores in BF16 at the same points
(weights, the input, every pre-activation, activation and pooled tensor;
the `out` layer is written in FP32), so that the forward pass can be
compared closely; the arithmetic stays FP64.
"""
import numpy as np
import torch
import torch.nn.functional as Fn

IN_PLANES = 8
LAYERS = [("e0a", IN_PLANES, 32), ("e0b", 32, 32), ("e1a", 32, 64), ("e1b", 64, 64),
          ("e2a", 64, 128), ("e2b", 128, 128), ("e3a", 128, 256), ("e3b", 256, 256),
          ("d2a", 256, 128), ("d2b", 128, 128), ("d1a", 128, 64), ("d1b", 64, 64),
          ("d0a", 64, 32), ("d0b", 32, 32), ("out", 32, 3)]


def layer_shapes():
    """(name, cout, cin) of every layer, in parameter order."""
    return [(name, co, ci) for name, ci, co in LAYERS]


def param_count():
    return sum(co * 9 * ci + co for _, ci, co in LAYERS)


def unpack(params):
    """Flat vector -> {name: (W [Cout][3][3][Cin], b)}."""
    return unpack_tensor(torch.as_tensor(np.asarray(params, dtype=np.float64)))


def conv3x3(h, w, b):
    """3 x 3 cross-correlation with zero padding 1: h [B][Cin][R][R],
    w [Cout][3][3][Cin], out[co][y][x] = b[co] + sum w[co][i][j][ci]
    h[ci][y + i - 1][x + j - 1]."""
    return Fn.conv2d(h, w.permute(0, 3, 1, 2), b, padding=1)


def _q(t, on):
    return t.to(torch.bfloat16).to(torch.float64) if on else t


def silu(z):
    return z * torch.sigmoid(z)


def forward_tensors(P, x, quantize=False):
    """Forward pass on torch tensors (P from `unpack`, x float64 B x 8 x R x R)."""
    q = lambda t: _q(t, quantize)  # noqa: E731

    def conv(h, name, skip=None):
        w, b = P[name]
        z = conv3x3(h, q(w), b)
        if skip is not None:
            z = z + skip
        return z

    def act(h, name, skip=None):
        return q(silu(q(conv(h, name, skip))))

    def pool(h):
        return q(Fn.avg_pool2d(h, 2))

    def up(h):
        return Fn.interpolate(h, scale_factor=2, mode="nearest")

    h = q(x)
    s0 = act(act(h, "e0a"), "e0b")
    s1 = act(act(pool(s0), "e1a"), "e1b")
    s2 = act(act(pool(s1), "e2a"), "e2b")
    h = act(act(pool(s2), "e3a"), "e3b")
    h = act(act(up(h), "d2a", s2), "d2b")
    h = act(act(up(h), "d1a", s1), "d1b")
    h = act(act(up(h), "d0a", s0), "d0b")
    return conv(h, "out")


def forward(params, x, quantize=False):
    """Network output (numpy float64, B x 3 x R x R)."""
    with torch.no_grad():
        P = unpack(params)
        y = forward_tensors(P, torch.as_tensor(np.asarray(x, dtype=np.float64)), quantize)
    return y.numpy()


def loss_and_grad(params, x, target):
    """Mean-square loss and its gradient with respect to the flat parameter
    vector (reverse-mode differentiation of the FP64 forward pass)."""
    p = torch.tensor(np.asarray(params, dtype=np.float64), requires_grad=True)
    P = unpack_tensor(p)
    y = forward_tensors(P, torch.as_tensor(np.asarray(x, dtype=np.float64)))
    loss = ((y - torch.as_tensor(np.asarray(target, dtype=np.float64))) ** 2).mean()
    loss.backward()
    return float(loss.detach()), p.grad.numpy().copy()


def unpack_tensor(p):
    """As `unpack`, keeping the autograd graph of the flat tensor p."""
    out, k = {}, 0
    for name, ci, co in LAYERS:
        w = p[k:k + co * 9 * ci].reshape(co, 3, 3, ci)
        k += co * 9 * ci
        out[name] = (w, p[k:k + co])
        k += co
    assert k == p.numel(), "parameter vector has %d entries, the network %d" % (p.numel(), k)
    return out


def loss(params, x, target):
    y = forward(params, x)
    return float(((y - np.asarray(target, dtype=np.float64)) ** 2).mean())
