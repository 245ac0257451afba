"""The C-ABI library loads and exports every entry point that include/mdf.h
declares; argument validation runs on the host and needs no GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2306_08216_gb300 import build as B
from paper_2306_08216_gb300 import mdf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mdf.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mdf.lib()


def declared_functions():
    text = "".join(open(os.path.join(ROOT, "include", h)).read() for h in sorted(os.listdir(os.path.join(ROOT, "include")))
                   if h.endswith(".h"))
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(mdf_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mdf_create", "mdf_step", "mdf_fields", "mdf_residual", "mdf_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert names, "no declarations parsed"
    for n in names:
        assert hasattr(lib, n), "libmdf.so does not export %s" % n
    assert sorted(mdf.exported_symbols()) == names


def test_library_links_no_torch(lib):
    # the boundary takes plain pointers; the library must not pull in torch
    out = os.popen("ldd %s" % mdf.LIB_PATH).read()
    # library names only (the load addresses are random hex and may contain "c10")
    names = [line.split()[0] for line in out.splitlines() if line.strip()]
    assert names and not any("torch" in n or n.startswith("libc10") for n in names), names


def _good():
    g = mdf.Grid(16, 16, 0, 1.0, 1.0)
    f = mdf.Fluid(0.01, 0, 0.0, 1.0, 0.0, 0.0)
    b = mdf.BC()
    p = mdf.Params(1.0, 0.5, 0.8, 1.5)
    return g, f, b, p


@pytest.mark.parametrize("mutate", [
    lambda g, f, b, p: setattr(g, "nx", 4),
    lambda g, f, b, p: setattr(g, "ny", 0),
    lambda g, f, b, p: setattr(g, "kind", 7),
    lambda g, f, b, p: setattr(g, "lx", 0.0),
    lambda g, f, b, p: setattr(f, "nu", -1.0),
    lambda g, f, b, p: setattr(f, "nu", float("nan")),
    lambda g, f, b, p: setattr(p, "cfl", 1.0),
    lambda g, f, b, p: setattr(p, "cfl", 0.0),
    lambda g, f, b, p: setattr(p, "eta", 1.5),
    lambda g, f, b, p: setattr(p, "c", 0.0),
    lambda g, f, b, p: setattr(p, "s_ratio", -1.0),
    lambda g, f, b, p: b.type.__setitem__(0, 1),          # west wall, east periodic
    lambda g, f, b, p: b.type.__setitem__(2, 5),
    lambda g, f, b, p: setattr(g, "kind", 1),             # separable grid without coordinates
    lambda g, f, b, p: (setattr(f, "power_law", 1), setattr(f, "K", 0.0)),
    lambda g, f, b, p: (setattr(f, "power_law", 1), setattr(f, "K", 1.0), setattr(f, "n", 1.0),
                        setattr(f, "nu_min", 2.0), setattr(f, "nu_max", 1.0)),
    lambda g, f, b, p: (setattr(g, "nx", 65536), setattr(g, "ny", 32769)),  # nx * ny > 2^31
    lambda g, f, b, p: setattr(p, "storage", 3),          # unknown storage mode
    lambda g, f, b, p: setattr(p, "storage", -1),
    # 16-bit storage with the alpha = 0 distribution
    lambda g, f, b, p: (setattr(p, "storage", 1), setattr(p, "rho0", 1)),
])
def test_invalid_arguments_rejected_before_any_cuda_call(lib, mutate):
    g, f, b, p = _good()
    mutate(g, f, b, p)
    st, msg = mdf.create_status(g, f, b, p)
    assert st == mdf.MDF_E_INVALID, (st, msg)
    assert msg


def test_null_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.mdf_create(None, None, None, None, ctypes.byref(h)) == mdf.MDF_E_INVALID
    assert lib.mdf_step(None, 1) == mdf.MDF_E_INVALID
    assert lib.mdf_residual(None, None, None) == mdf.MDF_E_INVALID
    assert lib.mdf_last_error(None)
    assert lib.mdf_steps_done(None) == -1
    assert lib.mdf_set_metrics(None, None, None, None, None, 0) == mdf.MDF_E_INVALID
    assert lib.mdf_residual_start(None) == mdf.MDF_E_INVALID
    assert lib.mdf_residual_finish(None, None, None) == mdf.MDF_E_INVALID


def test_creation_errors_are_per_thread(lib):
    """mdf_last_error(NULL) reports the calling thread's last failed create:
    thread A fails, thread B fails with another reason, then A reads A's."""
    import threading

    gate_a, gate_b = threading.Event(), threading.Event()
    seen = {}

    def a():
        g, f, b, p = _good()
        g.nx = 4
        h = ctypes.c_void_p()
        seen["a_st"] = lib.mdf_create(ctypes.byref(g), ctypes.byref(f), ctypes.byref(b), ctypes.byref(p),
                                      ctypes.byref(h))
        gate_a.set()
        gate_b.wait(30)
        seen["a"] = lib.mdf_last_error(None)

    def b_():
        gate_a.wait(30)
        g, f, b, p = _good()
        f.nu = -1.0
        h = ctypes.c_void_p()
        seen["b_st"] = lib.mdf_create(ctypes.byref(g), ctypes.byref(f), ctypes.byref(b), ctypes.byref(p),
                                      ctypes.byref(h))
        seen["b"] = lib.mdf_last_error(None)
        gate_b.set()

    ts = [threading.Thread(target=a), threading.Thread(target=b_)]
    for t in ts:
        t.start()
    for t in ts:
        t.join(60)
    assert seen["a_st"] == seen["b_st"] == mdf.MDF_E_INVALID
    assert b"nx" in seen["a"] and b"nu" in seen["b"], seen


def test_16bit_storage_passes_validation_on_every_grid_kind(lib):
    """16-bit storage is valid on curvilinear grids with walls and a power law
    (the tile kernel serves it): validation passes, and without a GPU the
    call fails only at the first CUDA call."""
    n = 16
    X, Y = np.meshgrid(np.arange(n) / n, np.arange(n) / n)
    g, f, b, p = mdf.problem_structs(n, n, grid="curvilinear", x=X + 0.05 * Y, y=Y, storage="fp16",
                                     walls=(True, True), power_law=(0.01, 0.8, 1e-4, 1.0))[:4]
    st, msg = mdf.create_status(g, f, b, p)
    assert st != mdf.MDF_E_INVALID, (st, msg)


def test_batch_rejects_mixed_storage(lib):
    g, f, b, p = _good()
    q = mdf.Params(1.0, 0.5, 0.8, 1.5, 1)
    G, F, B, P = (mdf.Grid * 2)(g, g), (mdf.Fluid * 2)(f, f), (mdf.BC * 2)(b, b), (mdf.Params * 2)(p, q)
    h = ctypes.c_void_p()
    assert lib.mdf_batch_create(2, G, F, B, P, ctypes.byref(h)) == mdf.MDF_E_INVALID
    assert b"same storage mode" in lib.mdf_batch_last_error(None)


def test_rho0_needs_fp32_storage(lib):
    g, f, b, p = mdf.problem_structs(16, 16, storage="bf16", rho0=True)[:4]
    st, msg = mdf.create_status(g, f, b, p)
    assert st == mdf.MDF_E_INVALID and "alpha = 0" in msg, (st, msg)


def test_batch_rejects_rho0(lib):
    g, f, b, p = _good()
    p.rho0 = 1
    G, F, B, P = (mdf.Grid * 2)(g, g), (mdf.Fluid * 2)(f, f), (mdf.BC * 2)(b, b), (mdf.Params * 2)(p, p)
    h = ctypes.c_void_p()
    assert lib.mdf_batch_create(2, G, F, B, P, ctypes.byref(h)) == mdf.MDF_E_INVALID
    assert b"rho_0" in lib.mdf_batch_last_error(None)


def test_empty_batch_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.mdf_batch_create(0, None, None, None, None, ctypes.byref(h)) == mdf.MDF_E_INVALID
    assert b"count" in lib.mdf_batch_last_error(None)


def test_launch_kind_calls_reject_null(lib):
    assert lib.mdf_launch_kind(None) == -1
    assert lib.mdf_batch_launch_kind(None) == -1
    assert lib.mdf_batch_set_launch(None, 1) == mdf.MDF_E_INVALID
    assert lib.mdf_set_launch(None, 0, 0) == mdf.MDF_E_INVALID
    assert lib.mdf_debug_poison(None) == mdf.MDF_E_INVALID


def test_rho0_calls_reject_null_contexts(lib):
    for fn in (lib.mdf_init_rho0, lib.mdf_get_rho0, lib.mdf_get_rho0_distributions,
               lib.mdf_set_rho0_distributions):
        assert fn(None, None, 0) == mdf.MDF_E_INVALID


def test_storage_names():
    assert mdf.STORAGE == {"fp32": 0, "fp16": 1, "bf16": 2}
    with pytest.raises(ValueError):
        mdf.problem_structs(8, 8, storage="fp8")


def test_net_create_rejects_bad_arguments_before_any_cuda_call(lib):
    h = ctypes.c_void_p()
    assert lib.mdf_net_create(12, 1, ctypes.byref(h)) == mdf.MDF_E_INVALID   # R % 8 != 0
    assert lib.mdf_net_create(8, 0, ctypes.byref(h)) == mdf.MDF_E_INVALID    # empty batch
    assert lib.mdf_net_create(16, 1, None) == mdf.MDF_E_INVALID
    assert lib.mdf_net_last_error(None)
    assert lib.mdf_net_param_count(None) == -1
