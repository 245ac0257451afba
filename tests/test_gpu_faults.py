"""Error paths of context creation, exercised by host-side fault injection
(MDF_FAIL_ALLOC=k fails the k-th allocation of a creation): every failing
creation returns MDF_E_NOMEM and frees what it allocated, and the library
keeps working afterwards.  No GPU fault is involved."""
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


@pytest.mark.parametrize("kind", ["uniform", "curvilinear", "batch"])
def test_every_failing_allocation_is_reported_and_released(kind):
    n = 65
    kw = dict(nu=0.01, walls=(True, True), u_wall=(0, 0, 0, 0.1))
    if kind == "curvilinear":
        X, Y = W.trapezoid_grid(n, n)
        kw.update(grid="curvilinear", x=X, y=Y)

    def make():
        if kind == "batch":
            return mdf.Batch([dict(nx=n, ny=n, **kw), dict(nx=33, ny=33, **kw)])
        return mdf.Solver(n, n, **kw)

    make().close()  # warm up the allocator and the kernels' attributes
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    try:
        for k in range(1, 60):
            os.environ["MDF_FAIL_ALLOC"] = str(k)
            try:
                obj = make()
            except mdf.MdfError as e:
                assert e.status == mdf.MDF_E_NOMEM, (k, e)
                failures += 1
                continue
            obj.close()  # k is past the last allocation: creation succeeded
            break
        else:
            pytest.fail("creation never succeeded")
    finally:
        os.environ.pop("MDF_FAIL_ALLOC", None)
    assert failures >= 8
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (4 << 20)  # nothing leaked
    s = mdf.Solver(n, n, **{k: v for k, v in kw.items()})
    s.init(*W.zeros(n, n))
    s.step(10)
    assert np.isfinite(s.state()).all()
