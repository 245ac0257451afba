"""Learned warm start: binding of the warm-start network (include/mdf_net.h)
and the pipeline around it.

The network predicts the steady state of a power-law lid-driven cavity from
(Re, n); the solver then marches from that prediction (mdf_init_fields) to
its own steady state, so the network only changes where the march starts.
The paper has no learned component; this is an extension of the library.

Every step runs in libmdf.so; this module marshals arguments, holds the
seeded training loop and moves fields between the network and the solver
on the device.
"""
import ctypes
import math
import os

import numpy as np

from . import mdf
from . import workloads as W

WEIGHTS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights")
U_LID = 0.1  # lid speed of the cavities the network is trained on


class Net:
    """The warm-start U-Net on R x R fields, batches of at most max_batch."""

    def __init__(self, resolution, max_batch, stream=None):
        L = mdf.lib()
        h = ctypes.c_void_p()
        st = L.mdf_net_create(resolution, max_batch, ctypes.byref(h))
        if st != mdf.MDF_OK:
            raise mdf.MdfError(st, L.mdf_net_last_error(None).decode())
        self._h = h
        self.R, self.max_batch = resolution, max_batch
        self.param_count = int(L.mdf_net_param_count(h))
        if stream is not None:
            raw = getattr(stream, "cuda_stream", stream)
            self._chk(L.mdf_net_set_stream(h, ctypes.c_void_p(raw or 0)))

    def _chk(self, st):
        if st != mdf.MDF_OK:
            raise mdf.MdfError(st, mdf.lib().mdf_net_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            mdf.lib().mdf_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layer_shapes(self):
        L = mdf.lib()
        out = []
        for k in range(L.mdf_net_layer_count(self._h)):
            s = (ctypes.c_int * 2)()
            self._chk(L.mdf_net_layer_shape(self._h, k, s))
            out.append((int(s[0]), int(s[1])))
        return out

    @staticmethod
    def _ptr(a):
        if hasattr(a, "data_ptr"):
            return ctypes.c_void_p(a.data_ptr()), 1
        return a.ctypes.data_as(ctypes.c_void_p), 0

    def set_params(self, p):
        if hasattr(p, "data_ptr"):
            assert p.numel() == self.param_count
            self._chk(mdf.lib().mdf_net_set_params(self._h, ctypes.c_void_p(p.data_ptr()), 1))
            return
        a = np.ascontiguousarray(p, dtype=np.float32)
        assert a.size == self.param_count, (a.size, self.param_count)
        self._chk(mdf.lib().mdf_net_set_params(self._h, a.ctypes.data_as(ctypes.c_void_p), 0))

    def get_params(self):
        a = np.empty(self.param_count, dtype=np.float32)
        self._chk(mdf.lib().mdf_net_get_params(self._h, a.ctypes.data_as(ctypes.c_void_p), 0))
        return a

    def _batch_args(self, inputs, targets=None):
        if hasattr(inputs, "data_ptr"):
            B = int(inputs.shape[0])
            assert inputs.is_contiguous() and tuple(inputs.shape[1:]) == (4, self.R, self.R)
            tp = ctypes.c_void_p(targets.data_ptr()) if targets is not None else None
            return B, ctypes.c_void_p(inputs.data_ptr()), tp, 1, (inputs, targets)
        x = np.ascontiguousarray(inputs, dtype=np.float32)
        assert x.shape[1:] == (4, self.R, self.R), x.shape
        t = None if targets is None else np.ascontiguousarray(targets, dtype=np.float32)
        tp = None if t is None else t.ctypes.data_as(ctypes.c_void_p)
        return x.shape[0], x.ctypes.data_as(ctypes.c_void_p), tp, 0, (x, t)

    def forward(self, inputs, out=None):
        """Outputs [B][3][R][R]: numpy for host inputs; for device (torch)
        inputs, written into `out` (a device tensor) or a new one."""
        B, xp, _, dev, keep = self._batch_args(inputs)
        if dev:
            import torch
            if out is None:
                out = torch.empty((B, 3, self.R, self.R), dtype=torch.float32, device=inputs.device)
            self._chk(mdf.lib().mdf_net_forward(self._h, B, xp, ctypes.c_void_p(out.data_ptr()), 1))
            return out
        y = np.empty((B, 3, self.R, self.R), dtype=np.float32)
        self._chk(mdf.lib().mdf_net_forward(self._h, B, xp, y.ctypes.data_as(ctypes.c_void_p), 0))
        return y

    def gradient(self, inputs, targets):
        B, xp, tp, dev, keep = self._batch_args(inputs, targets)
        g = np.empty(self.param_count, dtype=np.float32)
        loss = ctypes.c_double()
        if dev:
            import torch
            gd = torch.empty(self.param_count, dtype=torch.float32, device=inputs.device)
            self._chk(mdf.lib().mdf_net_gradient(self._h, B, xp, tp, ctypes.byref(loss),
                                                 ctypes.c_void_p(gd.data_ptr()), 1))
            return loss.value, gd.cpu().numpy()
        self._chk(mdf.lib().mdf_net_gradient(self._h, B, xp, tp, ctypes.byref(loss),
                                             g.ctypes.data_as(ctypes.c_void_p), 0))
        return loss.value, g

    def train_step(self, inputs, targets, lr, want_loss=True):
        B, xp, tp, dev, keep = self._batch_args(inputs, targets)
        loss = ctypes.c_double()
        self._chk(mdf.lib().mdf_net_train_step(self._h, B, xp, tp, float(lr),
                                               ctypes.byref(loss) if want_loss else None, dev))
        return loss.value if want_loss else None

    def save(self, path):
        np.save(path, self.get_params())

    def load(self, path):
        self.set_params(np.load(path))
