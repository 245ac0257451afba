"""Python binding of libmdf.so (include/mdf.h), argument marshalling only.

Every computation runs in the CUDA library; this module converts arguments
(numpy host arrays or torch CUDA tensors) into the C ABI's plain pointers.
There is no fallback: if libmdf.so is missing or cannot be loaded, importing
the binding's functions raises.

Low-level names mirror the C entry points (mdf_create, mdf_step, ...); the
``Solver`` class wraps one context with the keyword arguments of the problem
statement (grid, viscosity or power law, walls, forcing, scheme parameters).
"""
import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# MDF_DEBUG_LIBRARY=1 loads the debug build (libmdf_debug.so, index checks)
LIB_PATH = os.path.join(HERE, "libmdf_debug.so" if os.environ.get("MDF_DEBUG_LIBRARY") == "1" else "libmdf.so")

MDF_OK, MDF_E_INVALID, MDF_E_CUDA, MDF_E_NOMEM, MDF_E_DIVERGED, MDF_E_TIMEOUT, MDF_E_STATE = range(7)
STATUS_NAMES = {0: "MDF_OK", 1: "MDF_E_INVALID", 2: "MDF_E_CUDA", 3: "MDF_E_NOMEM",
                4: "MDF_E_DIVERGED", 5: "MDF_E_TIMEOUT", 6: "MDF_E_STATE"}
GRID_KINDS = {"uniform": 0, "separable": 1, "curvilinear": 2}
FIELD_NAMES = ["u", "v", "P", "dudx", "dudy", "dvdx", "dvdy", "div",
               "Sxx", "Sxy", "Syy", "sigma_xx", "sigma_xy", "sigma_yy",
               "Omega_xy", "vorticity", "nu"]

_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)


class MdfError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("kind", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("x", _D), ("y", _D)]


class Fluid(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("power_law", ctypes.c_int), ("K", ctypes.c_double),
                ("n", ctypes.c_double), ("nu_min", ctypes.c_double), ("nu_max", ctypes.c_double)]


class BC(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int * 4), ("u_wall", ctypes.c_double * 4), ("v_wall", ctypes.c_double * 4)]


class Params(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double), ("cfl", ctypes.c_double), ("eta", ctypes.c_double),
                ("s_ratio", ctypes.c_double), ("storage", ctypes.c_int), ("rho0", ctypes.c_int)]


# mdf_params.storage: how the state is kept between steps (arithmetic is FP32)
STORAGE = {"fp32": 0, "fp16": 1, "bf16": 2}


# (name, restype, argtypes) of every entry point declared in include/*.h
_SIGNATURES = [
    ("mdf_create", ctypes.c_int, [ctypes.POINTER(Grid), ctypes.POINTER(Fluid), ctypes.POINTER(BC),
                                  ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_void_p)]),
    ("mdf_destroy", None, [ctypes.c_void_p]),
    ("mdf_set_stream", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("mdf_set_force", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("mdf_set_force_rate", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("mdf_set_source", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p,
                                      ctypes.c_int]),
    ("mdf_set_metrics", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int]),
    ("mdf_init_fields", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int]),
    ("mdf_init_rho0", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("mdf_get_rho0", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("mdf_get_rho0_distributions", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("mdf_set_rho0_distributions", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("mdf_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("mdf_fields", ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]),
    ("mdf_residual", ctypes.c_int, [ctypes.c_void_p, _D, _D]),
    ("mdf_residual_start", ctypes.c_int, [ctypes.c_void_p]),
    ("mdf_residual_finish", ctypes.c_int, [ctypes.c_void_p, _D, _D]),
    ("mdf_get_distributions", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("mdf_set_distributions", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("mdf_synchronize", ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    ("mdf_save", ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    ("mdf_load", ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    ("mdf_dt", ctypes.c_double, [ctypes.c_void_p]),
    ("mdf_steps_done", ctypes.c_longlong, [ctypes.c_void_p]),
    ("mdf_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("mdf_launch_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    ("mdf_set_launch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("mdf_launch_kind", ctypes.c_int, [ctypes.c_void_p]),
    ("mdf_debug_poison", ctypes.c_int, [ctypes.c_void_p]),
    ("mdf_bytes_per_node", ctypes.c_double, [ctypes.c_void_p]),
    ("mdf_batch_create", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Grid), ctypes.POINTER(Fluid),
                                        ctypes.POINTER(BC), ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_void_p)]),
    ("mdf_batch_destroy", None, [ctypes.c_void_p]),
    ("mdf_batch_set_stream", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("mdf_batch_init_fields", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_int]),
    ("mdf_batch_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("mdf_batch_residual", ctypes.c_int, [ctypes.c_void_p, _D, ctypes.POINTER(ctypes.c_int)]),
    ("mdf_batch_problem", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    ("mdf_batch_set_active", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    ("mdf_batch_info", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)]),
    ("mdf_batch_set_launch", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("mdf_batch_launch_kind", ctypes.c_int, [ctypes.c_void_p]),
    ("mdf_batch_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("mdf_residual_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p]),
    # include/mdf_net.h (warm-start network)
    ("mdf_net_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    ("mdf_net_destroy", None, [ctypes.c_void_p]),
    ("mdf_net_set_stream", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("mdf_net_set_conv_kernel", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("mdf_net_param_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("mdf_net_layer_count", ctypes.c_int, [ctypes.c_void_p]),
    ("mdf_net_layer_shape", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    ("mdf_net_set_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("mdf_net_get_params", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("mdf_net_forward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_int]),
    ("mdf_net_gradient", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, _D,
                                        ctypes.c_void_p, ctypes.c_int]),
    ("mdf_net_train_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                          ctypes.c_double, _D, ctypes.c_int]),
    ("mdf_net_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
]

_lib = None


def lib():
    """Load libmdf.so (built by ``paper_2306_08216_gb300.build``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("%s is not built; run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in _SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return [s[0] for s in _SIGNATURES]


def _check(status, ctx=None):
    if status != MDF_OK:
        msg = lib().mdf_last_error(ctx)
        raise MdfError(status, msg.decode() if msg else "")


def _is_torch_cuda(a):
    return hasattr(a, "is_cuda") and a.is_cuda


class _Arr:
    """A float32 argument as a pointer plus its on_device flag; keeps the
    backing object alive."""

    def __init__(self, a, n=None):
        if _is_torch_cuda(a):
            import torch
            assert a.dtype == torch.float32 and a.is_contiguous()
            self.obj = a
            self.ptr = ctypes.c_void_p(a.data_ptr())
            self.on_device = 1
        else:
            self.obj = np.ascontiguousarray(a, dtype=np.float32)
            self.ptr = self.obj.ctypes.data_as(ctypes.c_void_p)
            self.on_device = 0
        if n is not None:
            size = a.numel() if self.on_device else self.obj.size
            assert size == n, "expected %d elements, got %d" % (n, size)


def problem_structs(nx, ny, nu=0.01, grid="uniform", lx=1.0, ly=1.0, x=None, y=None, power_law=None,
                    walls=(False, False), u_wall=(0, 0, 0, 0), v_wall=(0, 0, 0, 0), c=1.0, cfl=0.5, eta=0.8,
                    s_ratio=1.5, storage="fp32", rho0=False):
    """The C structs (mdf_grid, mdf_fluid, mdf_bc, mdf_params) of one problem,
    plus the arrays they point to (keep them alive while the structs are used)."""
    keep = []
    g = Grid(nx, ny, GRID_KINDS[grid], lx, ly)
    if grid != "uniform":
        xa = np.ascontiguousarray(x, dtype=np.float64).ravel()
        ya = np.ascontiguousarray(y, dtype=np.float64).ravel()
        keep += [xa, ya]
        g.x, g.y = xa.ctypes.data_as(_D), ya.ctypes.data_as(_D)
    f = Fluid(nu, 0, 0.0, 1.0, 0.0, 0.0)
    if power_law is not None:
        f.power_law = 1
        f.K, f.n, f.nu_min, f.nu_max = power_law
    b = BC()
    for k in range(4):
        b.type[k] = 1 if walls[0 if k < 2 else 1] else 0
        b.u_wall[k] = u_wall[k]
        b.v_wall[k] = v_wall[k]
    if storage not in STORAGE:
        raise ValueError("storage must be one of %s" % sorted(STORAGE))
    p = Params(c, cfl, eta, s_ratio, STORAGE[storage], 1 if rho0 else 0)
    return g, f, b, p, keep


class Solver:
    """One MDF-FDLBM problem on the GPU (see include/mdf.h).

    Keyword arguments are those of the test oracle: nx, ny, nu, grid
    ("uniform" | "separable" | "curvilinear"), lx, ly, x, y, power_law
    (K, n, nu_min, nu_max), walls (x_walls, y_walls), u_wall, v_wall
    (west, east, south, north), c, cfl, eta, s_ratio, force (None, (fx, fy)
    constants or (Fx, Fy) fields), and storage ("fp32", or "fp16" / "bf16":
    u, v, P in FP32 plus the non-equilibrium part in 16 bits; periodic
    Newtonian problems on uniform or separable grids only), force_rate,
    source, and rho0 (True: also evolve the alpha = 0 distribution of
    Eq. 2.1.2, which starts at rho_0 = 1; FP32 storage only).
    """

    def __init__(self, nx, ny, nu=0.01, grid="uniform", lx=1.0, ly=1.0, x=None, y=None,
                 power_law=None, walls=(False, False), u_wall=(0, 0, 0, 0), v_wall=(0, 0, 0, 0),
                 c=1.0, cfl=0.5, eta=0.8, s_ratio=1.5, force=None, stream=None, storage="fp32", force_rate=None,
                 source=None, rho0=False, _handle=None):
        self.nx, self.ny = nx, ny
        self._owned = _handle is None
        if _handle is not None:  # a problem of a batch: the batch owns the context
            self._h = _handle
            return
        g, f, b, p, self._keep = problem_structs(nx, ny, nu, grid, lx, ly, x, y, power_law, walls, u_wall, v_wall,
                                                 c, cfl, eta, s_ratio, storage, rho0)
        h = ctypes.c_void_p()
        _check(lib().mdf_create(ctypes.byref(g), ctypes.byref(f), ctypes.byref(b), ctypes.byref(p), ctypes.byref(h)))
        self._h = h
        if stream is not None:
            self.set_stream(stream)
        if force is not None:
            self.set_force(force)
        if force_rate is not None:
            self.set_force_rate(force_rate)
        if source is not None:
            self.set_source(source)

    def close(self):
        if getattr(self, "_h", None) and getattr(self, "_owned", True):
            lib().mdf_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def dt(self):
        return lib().mdf_dt(self._h)

    @property
    def steps(self):
        return lib().mdf_steps_done(self._h)

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
        raw = getattr(stream, "cuda_stream", stream)
        _check(lib().mdf_set_stream(self._h, ctypes.c_void_p(raw or 0)), self._h)

    def set_force(self, force):
        if force is None:
            _check(lib().mdf_set_force(self._h, 0, 0.0, 0.0, None, None, 0), self._h)
        elif np.isscalar(force[0]):
            _check(lib().mdf_set_force(self._h, 1, float(force[0]), float(force[1]), None, None, 0), self._h)
        else:
            n = self.nx * self.ny
            fx, fy = _Arr(force[0], n), _Arr(force[1], n)
            _check(lib().mdf_set_force(self._h, 2, 0.0, 0.0, fx.ptr, fy.ptr, fx.on_device), self._h)
            self.synchronize()

    def set_force_rate(self, rate):
        """dF/dt of the body force (None, (dfx, dfy) or fields), Eq. 2.3.24."""
        if rate is None:
            _check(lib().mdf_set_force_rate(self._h, 0, 0.0, 0.0, None, None, 0), self._h)
        elif np.isscalar(rate[0]):
            _check(lib().mdf_set_force_rate(self._h, 1, float(rate[0]), float(rate[1]), None, None, 0), self._h)
        else:
            n = self.nx * self.ny
            fx, fy = _Arr(rate[0], n), _Arr(rate[1], n)
            _check(lib().mdf_set_force_rate(self._h, 2, 0.0, 0.0, fx.ptr, fy.ptr, fx.on_device), self._h)
            self.synchronize()

    def set_source(self, R):
        """Source R of div u = R (None, a constant or a field), Eq. 2.3.23."""
        if R is None:
            _check(lib().mdf_set_source(self._h, 0, 0.0, None, 0), self._h)
        elif np.isscalar(R):
            _check(lib().mdf_set_source(self._h, 1, float(R), None, 0), self._h)
        else:
            a = _Arr(R, self.nx * self.ny)
            _check(lib().mdf_set_source(self._h, 2, 0.0, a.ptr, a.on_device), self._h)
            self.synchronize()

    def set_metrics(self, xi_x, xi_y, eta_x, eta_y):
        """Metric coefficients of a curvilinear grid (FP64, ny x nx each, per
        unit node index) in place of those differenced from the coordinates."""
        n = self.nx * self.ny
        arrs = [np.ascontiguousarray(m, dtype=np.float64).ravel() for m in (xi_x, xi_y, eta_x, eta_y)]
        for a in arrs:
            assert a.size == n, "expected %d elements, got %d" % (n, a.size)
        ptrs = [a.ctypes.data_as(ctypes.c_void_p) for a in arrs]
        _check(lib().mdf_set_metrics(self._h, *ptrs, 0), self._h)

    def init(self, u, v, p):
        n = self.nx * self.ny
        a = [_Arr(t, n) for t in (u, v, p)]
        _check(lib().mdf_init_fields(self._h, a[0].ptr, a[1].ptr, a[2].ptr, a[0].on_device), self._h)
        if a[0].on_device:
            self.synchronize()

    def init_rho0(self, rho0):
        """fhat_{j,0} = feq_{j,0}(rho0, u) with u of the current state."""
        a = _Arr(rho0, self.nx * self.ny)
        _check(lib().mdf_init_rho0(self._h, a.ptr, a.on_device), self._h)
        if a.on_device:
            self.synchronize()

    def rho0(self):
        """rho_0 = sum_j fhat_{j,0} as float32 [ny, nx]."""
        out = np.empty((self.ny, self.nx), dtype=np.float32)
        _check(lib().mdf_get_rho0(self._h, out.ctypes.data_as(ctypes.c_void_p), 0), self._h)
        return out

    def rho0_state(self):
        """fhat_{j,0} as float32 [5, ny, nx]."""
        out = np.empty((5, self.ny, self.nx), dtype=np.float32)
        _check(lib().mdf_get_rho0_distributions(self._h, out.ctypes.data_as(ctypes.c_void_p), 0), self._h)
        return out

    def set_rho0_state(self, g):
        a = _Arr(g, 5 * self.nx * self.ny)
        _check(lib().mdf_set_rho0_distributions(self._h, a.ptr, a.on_device), self._h)
        if a.on_device:
            self.synchronize()

    def step(self, n=1):
        _check(lib().mdf_step(self._h, int(n)), self._h)

    def synchronize(self, timeout=0.0):
        _check(lib().mdf_synchronize(self._h, float(timeout)), self._h)

    def state(self, out=None):
        """fhat as float32 [2, 5, ny, nx]; `out` may be a torch CUDA tensor."""
        if out is not None and _is_torch_cuda(out):
            _check(lib().mdf_get_distributions(self._h, ctypes.c_void_p(out.data_ptr()), 1), self._h)
            return out
        arr = np.empty((2, 5, self.ny, self.nx), dtype=np.float32)
        _check(lib().mdf_get_distributions(self._h, arr.ctypes.data_as(ctypes.c_void_p), 0), self._h)
        return arr

    def set_state(self, fh):
        a = _Arr(fh, 10 * self.nx * self.ny)
        _check(lib().mdf_set_distributions(self._h, a.ptr, a.on_device), self._h)

    def fields(self, names=None, out=None):
        """Derived fields as float32 [ny, nx] host arrays, by name.  `out`
        (optional) maps names to caller-owned C-contiguous float32 host
        arrays of that shape -- numpy arrays or CPU torch tensors, e.g. in
        pinned memory, which the device copies into directly -- and is
        filled and returned in their place."""
        names = FIELD_NAMES if names is None else list(names)
        mask = 0
        for nm in names:
            mask |= 1 << FIELD_NAMES.index(nm)
        order = [nm for nm in FIELD_NAMES if mask & (1 << FIELD_NAMES.index(nm))]
        outs = []
        for nm in order:
            o = None if out is None else out.get(nm)
            if o is None:
                o = np.empty((self.ny, self.nx), dtype=np.float32)
            elif not isinstance(o, np.ndarray):
                assert not _is_torch_cuda(o), "fields(out=...) takes host arrays"
                o = o.numpy()
            assert o.dtype == np.float32 and o.shape == (self.ny, self.nx) and o.flags["C_CONTIGUOUS"], \
                "out[%r] must be a C-contiguous float32 array of shape %s" % (nm, (self.ny, self.nx))
            outs.append(o)
        ptrs = (ctypes.c_void_p * len(outs))(*[o.ctypes.data_as(ctypes.c_void_p) for o in outs])
        _check(lib().mdf_fields(self._h, mask, ptrs, 0), self._h)
        res = dict(zip(order, outs))
        if out is not None:
            for nm in order:
                if nm in out and not isinstance(out[nm], np.ndarray):
                    res[nm] = out[nm]
        return res

    def fields_device(self, outs):
        """outs: dict name -> float32 CUDA tensor (ny, nx); asynchronous."""
        mask = 0
        for nm in outs:
            mask |= 1 << FIELD_NAMES.index(nm)
        order = [nm for nm in FIELD_NAMES if mask & (1 << FIELD_NAMES.index(nm))]
        ptrs = (ctypes.c_void_p * len(order))(*[ctypes.c_void_p(outs[nm].data_ptr()) for nm in order])
        _check(lib().mdf_fields(self._h, mask, ptrs, 1), self._h)

    def residual(self):
        """(r, (sum u, sum v)); raises MdfError on divergence."""
        r = ctypes.c_double()
        d = (ctypes.c_double * 2)()
        st = lib().mdf_residual(self._h, ctypes.byref(r), d)
        if st not in (MDF_OK,):
            _check(st, self._h)
        return r.value, (d[0], d[1])

    def residual_start(self):
        """Enqueue a residual check; collect it with residual_finish()."""
        _check(lib().mdf_residual_start(self._h), self._h)

    def residual_finish(self):
        """(r, (sum u, sum v)) of the check residual_start() enqueued; waits
        for that work only.  Raises MdfError on divergence."""
        r = ctypes.c_double()
        d = (ctypes.c_double * 2)()
        _check(lib().mdf_residual_finish(self._h, ctypes.byref(r), d), self._h)
        return r.value, (d[0], d[1])

    def save(self, path):
        _check(lib().mdf_save(self._h, str(path).encode()), self._h)

    def load(self, path):
        _check(lib().mdf_load(self._h, str(path).encode()), self._h)

    def launch_info(self):
        info = (ctypes.c_int * 8)()
        _check(lib().mdf_launch_info(self._h, info), self._h)
        keys = ["threads", "cols_per_block", "rows_per_block", "grid_x", "grid_y", "smem_bytes",
                "blocks_per_sm", "pitch"]
        d = dict(zip(keys, list(info)))
        d["kernel"] = "tile" if lib().mdf_launch_kind(self._h) == 1 else "march"
        return d

    def set_launch(self, threads, rows_per_block=0):
        """threads 128 / 256: a march plan with that block size and band
        height; threads 0: the 16 x 16 tile kernel."""
        _check(lib().mdf_set_launch(self._h, int(threads), int(rows_per_block)), self._h)

    def bytes_per_node(self):
        return lib().mdf_bytes_per_node(self._h)

    def debug_poison(self):
        """NaN into the storage no valid result may read (see mdf_debug_poison)."""
        _check(lib().mdf_debug_poison(self._h), self._h)


def create_status(grid, fluid, bc, params=None):
    """Call mdf_create with raw structs; returns (status, message).  Used to
    check argument validation, which happens before any CUDA call."""
    L = lib()
    h = ctypes.c_void_p()
    st = L.mdf_create(ctypes.byref(grid), ctypes.byref(fluid), ctypes.byref(bc),
                      ctypes.byref(params) if params is not None else None, ctypes.byref(h))
    msg = L.mdf_last_error(None)
    if st == MDF_OK:
        L.mdf_destroy(h)
    return st, (msg.decode() if msg else "")


class Batch:
    """Many problems advanced by one persistent launch per time step
    (mdf_batch_*).  `problems` is a list of keyword dicts as for Solver
    (without stream/force); problem i is available as batch.problem(i), a
    Solver view on the batch's context (no step(); the batch steps it)."""

    def __init__(self, problems, stream=None):
        L = lib()
        n = len(problems)
        G, F, B, P = (Grid * n)(), (Fluid * n)(), (BC * n)(), (Params * n)()
        self._keep = []
        for i, kw in enumerate(problems):
            kw = dict(kw)
            nx, ny = kw.pop("nx"), kw.pop("ny")
            g, f, b, p, keep = problem_structs(nx, ny, **kw)
            G[i], F[i], B[i], P[i] = g, f, b, p
            self._keep += keep
        h = ctypes.c_void_p()
        st = L.mdf_batch_create(n, G, F, B, P, ctypes.byref(h))
        if st != MDF_OK:
            raise MdfError(st, L.mdf_batch_last_error(None).decode())
        self._h = h
        self.count = n
        self.shapes = [(kw["nx"], kw["ny"]) for kw in problems]
        if stream is not None:
            raw = getattr(stream, "cuda_stream", stream)
            self._chk(L.mdf_batch_set_stream(self._h, ctypes.c_void_p(raw or 0)))

    def _chk(self, st):
        if st != MDF_OK:
            raise MdfError(st, lib().mdf_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().mdf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, index, u, v, p):
        nx, ny = self.shapes[index]
        a = [_Arr(t, nx * ny) for t in (u, v, p)]
        self._chk(lib().mdf_batch_init_fields(self._h, index, a[0].ptr, a[1].ptr, a[2].ptr, a[0].on_device))

    def step(self, n=1):
        self._chk(lib().mdf_batch_step(self._h, int(n)))

    def residual(self):
        """(residuals[count], statuses[count]); divergence is reported in the
        statuses, not raised."""
        r = (ctypes.c_double * self.count)()
        s = (ctypes.c_int * self.count)()
        st = lib().mdf_batch_residual(self._h, r, s)
        if st not in (MDF_OK, MDF_E_DIVERGED):
            self._chk(st)
        return np.array(r[:]), np.array(s[:])

    def set_active(self, index, active):
        """Retire (False) or re-admit (True) problem `index`."""
        self._chk(lib().mdf_batch_set_active(self._h, int(index), 1 if active else 0))

    def problem(self, index):
        h = ctypes.c_void_p()
        self._chk(lib().mdf_batch_problem(self._h, index, ctypes.byref(h)))
        nx, ny = self.shapes[index]
        return Solver(nx, ny, _handle=h)

    def info(self):
        v = (ctypes.c_longlong * 6)()
        self._chk(lib().mdf_batch_info(self._h, v))
        d = dict(zip(["problems", "work_items", "blocks", "blocks_per_sm", "nodes", "steps"], list(v)))
        d["kernel"] = {0: "march", 1: "tile", 2: "march_rolled"}[lib().mdf_batch_launch_kind(self._h)]
        return d

    def set_launch(self, kernel):
        """kernel: "march" (strips x bands per problem), "march_rolled" (the same
        march in rolled form) or "tile" (16 x 16 tiles)."""
        self._chk(lib().mdf_batch_set_launch(self._h, {"march": 0, "tile": 1, "march_rolled": 2}[kernel]))
