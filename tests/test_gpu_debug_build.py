"""The debug build (libmdf_debug.so, -DMDF_DEBUG): the step kernels check
the index of every global load and store that does not go through TMA (the
state stores of every kernel, the tile kernel's state loads, force and
source fields), skip one outside its buffer and raise an error word that the
next host wait turns into MDF_E_CUDA -- a bounds checker that cannot fault
the GPU.  Every kernel family and storage mode steps a small ragged case
through it (in a child process, since one process loads one library): no
check fires, and the states equal those of the release build to the bit
(the checks change no arithmetic)."""
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2306_08216_gb300 import build as B  # noqa: E402

B.build()
HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_runs_every_kernel_family_clean_and_bitwise(tmp_path):
    B.build(debug=True)
    import debug_cases as D  # noqa: E402 (tests/ is on sys.path under pytest)

    release = D.run_cases()
    out = tmp_path / "debug.npz"
    env = dict(os.environ, MDF_DEBUG_LIBRARY="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_cases.py"), str(out)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    debug = np.load(out)
    assert str(debug["library"]) == "libmdf_debug.so"
    assert sorted(k for k in debug.files if k != "library") == sorted(release)
    for k, v in release.items():
        np.testing.assert_array_equal(debug[k], v, err_msg=k)
