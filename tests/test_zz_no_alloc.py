"""mdf_residual_noalloc: the residual/drift reduction for callers that may
not allocate device memory -- code running under an allocator that owns all
device memory and forbids side allocations, or in a loop that must not risk
an allocation failure or the device-wide synchronisation that cudaMalloc
and cudaFree imply.  It must agree with mdf_residual, the entry point that
reduces through its context's allocated scratch, on two calls in a row, at
a small size and at the largest size its fixed scratch serves, and a call
must leave the device's memory use unchanged.

This file is collected last so that a run stopping at the first failure has
already run every other test.
"""
import ctypes
import math

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


def noalloc(fhat, u_prev, v_prev, nx, ny, window, stream, out):
    return mdf.lib().mdf_residual_noalloc(
        ctypes.c_void_p(fhat.data_ptr()), ctypes.c_void_p(u_prev.data_ptr()), ctypes.c_void_p(v_prev.data_ptr()),
        nx, ny, window, ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(out.data_ptr()))


@pytest.mark.parametrize("n", [96, 4096])
def test_noalloc_residual_matches_mdf_residual_twice(n):
    """Taylor-Green on n x n nodes (4096^2 fills every one of the fixed
    scratch's partial-sum slots); two windows of K steps in a row."""
    U0, K = 0.01, 40
    stream = torch.cuda.Stream()
    s = mdf.Solver(n, n, nu=0.01, lx=2 * math.pi, ly=2 * math.pi, stream=stream)
    s.init(*W.taylor_green(n, U0))
    fhat = torch.empty((2, 5, n, n), dtype=torch.float32, device="cuda")
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    prev = {k: torch.empty((n, n), dtype=torch.float32, device="cuda") for k in ("u", "v")}
    for call in range(2):
        s.fields_device(prev)
        s.step(K)
        s.state(out=fhat)
        stream.synchronize()
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        st = noalloc(fhat, prev["u"], prev["v"], n, n, K, stream, out)
        assert st == mdf.MDF_OK
        stream.synchronize()
        if call == 1:  # the first call may load the kernels' module
            assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_allocated() == alloc0
        r_ref, drift_ref = s.residual()   # the existing entry point, same window
        got = out.cpu().numpy()
        assert np.isfinite(got[0]) and got[3] == 0.0
        assert got[0] == pytest.approx(r_ref, rel=1e-10), call
        tol = 1e-12 * float(np.abs(prev["u"].cpu().numpy()).sum()) + 1e-18
        assert abs(got[1] - drift_ref[0]) <= tol and abs(got[2] - drift_ref[1]) <= tol, call
    s.close()


def test_noalloc_rejects_fields_larger_than_its_static_scratch():
    t = torch.empty(16, dtype=torch.float32, device="cuda")
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    assert noalloc(t, t, t, 4097, 4096, 1, stream, out) == mdf.MDF_E_INVALID
    assert noalloc(t, t, t, 8, 8, 0, stream, out) == mdf.MDF_E_INVALID
