"""ctypes wrapper of the FP64 CPU oracle (``mdf_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the CPU-baseline leg of ``bench.py``; never by the library.  It shares no code
with the CUDA path.  See ``mdf_oracle.c`` for the method (arXiv:2306.08216,
Sec. 2.2 Steps (1)-(4)) and the readings it takes.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mdf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_mdf.so")

FIELD_NAMES = ["u", "v", "P", "dudx", "dudy", "dvdx", "dvdy", "div",
               "Sxx", "Sxy", "Syy", "sigma_xx", "sigma_xy", "sigma_yy",
               "Omega_xy", "vorticity", "nu"]

_D = ctypes.POINTER(ctypes.c_double)


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("grid_kind", ctypes.c_int),
        ("lx", ctypes.c_double), ("ly", ctypes.c_double),
        ("xc", _D), ("yc", _D),
        ("nu", ctypes.c_double),
        ("power_law", ctypes.c_int),
        ("K", ctypes.c_double), ("n_index", ctypes.c_double),
        ("nu_min", ctypes.c_double), ("nu_max", ctypes.c_double),
        ("bc", ctypes.c_int * 4),
        ("u_wall", ctypes.c_double * 4), ("v_wall", ctypes.c_double * 4),
        ("c", ctypes.c_double), ("cfl", ctypes.c_double),
        ("eta", ctypes.c_double), ("s_ratio", ctypes.c_double),
        ("force_mode", ctypes.c_int),
        ("fx", ctypes.c_double), ("fy", ctypes.c_double),
        ("force_x", _D), ("force_y", _D),
        ("threads", ctypes.c_int),
        ("rho0", ctypes.c_int),
    ]


def build(force=False):
    """Compile the oracle with gcc (plain C99 + OpenMP, IEEE arithmetic)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-std=gnu99", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
           "-shared", "-fPIC", "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.POINTER(OrcParams)]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_last_status.restype = ctypes.c_int
        L.orc_dt.restype = ctypes.c_double
        L.orc_dt.argtypes = [ctypes.c_void_p]
        L.orc_cs2.restype = ctypes.c_double
        L.orc_cs2.argtypes = [ctypes.c_void_p]
        L.orc_steps.restype = ctypes.c_long
        L.orc_steps.argtypes = [ctypes.c_void_p]
        L.orc_init.argtypes = [ctypes.c_void_p, _D, _D, _D]
        L.orc_set_state.argtypes = [ctypes.c_void_p, _D]
        L.orc_get_state.argtypes = [ctypes.c_void_p, _D]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
        L.orc_fields.argtypes = [ctypes.c_void_p, _D]
        L.orc_collision_matrix.argtypes = [ctypes.c_void_p, ctypes.c_double, _D]
        L.orc_lambda_matrix.argtypes = [ctypes.c_void_p, _D]
        L.orc_max_threads.restype = ctypes.c_int
        L.orc_set_force.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _D]
        L.orc_set_force_rate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D, _D]
        for fn in ("orc_init_rho0", "orc_rho0", "orc_get_rho0_state", "orc_set_rho0_state"):
            getattr(L, fn).restype = ctypes.c_int
            getattr(L, fn).argtypes = [ctypes.c_void_p, _D]
        L.orc_set_source.restype = ctypes.c_int
        L.orc_set_source.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, _D]
        L.orc_set_metrics.restype = ctypes.c_int
        L.orc_set_metrics.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
        L.orc_get_metrics.restype = ctypes.c_int
        L.orc_get_metrics.argtypes = [ctypes.c_void_p, _D, _D, _D, _D]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_D)


class Oracle:
    """One MDF-FDLBM problem stepped in FP64 on the host.

    Keyword arguments mirror the library's problem statement:
      nx, ny            nodes per axis
      grid              "uniform" (lx, ly), "separable" (x[nx], y[ny]) or
                        "curvilinear" (x[ny,nx], y[ny,nx]); periodic axes of
                        the last two need lx / ly as the period
      nu                kinematic viscosity (Newtonian)
      power_law         (K, n, nu_min, nu_max) or None
      walls             (x_walls, y_walls) booleans; walls are NEE velocity walls
      u_wall, v_wall    4-tuples, west/east/south/north
      c, cfl, eta, s_ratio  lattice speed, CFL number, mixed-scheme weight, s'/s
      force             None, (fx, fy) constants, or (Fx[ny,nx], Fy[ny,nx])
      force_rate        dF/dt in the same forms (Eq. 2.3.24)
      source            R of Eq. 2.1.1: None, a constant or R[ny,nx]
      rho0              also evolve the alpha = 0 distribution (rho_0, Eq. 2.1.2)
    """

    def __init__(self, nx, ny, nu=0.01, grid="uniform", lx=1.0, ly=1.0, x=None, y=None,
                 power_law=None, walls=(False, False), u_wall=(0, 0, 0, 0),
                 v_wall=(0, 0, 0, 0), c=1.0, cfl=0.5, eta=0.8, s_ratio=1.5,
                 force=None, force_rate=None, source=None, rho0=False, threads=0):
        L = lib()
        p = OrcParams()
        p.nx, p.ny = nx, ny
        p.grid_kind = {"uniform": 0, "separable": 1, "curvilinear": 2}[grid]
        p.lx, p.ly = lx, ly
        self._keep = []
        if grid != "uniform":
            xa = np.ascontiguousarray(x, dtype=np.float64).ravel()
            ya = np.ascontiguousarray(y, dtype=np.float64).ravel()
            self._keep += [xa, ya]
            p.xc, p.yc = _ptr(xa), _ptr(ya)
        p.nu = nu
        if power_law is not None:
            p.power_law = 1
            p.K, p.n_index, p.nu_min, p.nu_max = power_law
        p.bc[0] = p.bc[1] = 1 if walls[0] else 0
        p.bc[2] = p.bc[3] = 1 if walls[1] else 0
        for k in range(4):
            p.u_wall[k] = u_wall[k]
            p.v_wall[k] = v_wall[k]
        p.c, p.cfl, p.eta, p.s_ratio = c, cfl, eta, s_ratio
        if force is None:
            p.force_mode = 0
        elif np.isscalar(force[0]):
            p.force_mode = 1
            p.fx, p.fy = float(force[0]), float(force[1])
        else:
            p.force_mode = 2
            fxa = np.ascontiguousarray(force[0], dtype=np.float64).ravel()
            fya = np.ascontiguousarray(force[1], dtype=np.float64).ravel()
            self._keep += [fxa, fya]
            p.force_x, p.force_y = _ptr(fxa), _ptr(fya)
        p.threads = threads
        p.rho0 = 1 if rho0 else 0
        self._p = p
        h = L.orc_create(ctypes.byref(p))
        if not h:
            raise ValueError("oracle rejected the parameters (status %d)" % L.orc_last_status())
        self._h = h
        self.nx, self.ny = nx, ny
        if force_rate is not None:
            self.set_force_rate(force_rate)
        if source is not None:
            self.set_source(source)

    @staticmethod
    def _pair(pair):
        if pair is None:
            return 0, 0.0, 0.0, None, None, []
        if np.isscalar(pair[0]):
            return 1, float(pair[0]), float(pair[1]), None, None, []
        a = np.ascontiguousarray(pair[0], dtype=np.float64).ravel()
        b = np.ascontiguousarray(pair[1], dtype=np.float64).ravel()
        return 2, 0.0, 0.0, _ptr(a), _ptr(b), [a, b]

    def set_force(self, force):
        """Replace the body force (None, (fx, fy) or fields) before the next step."""
        m, a, b, pa, pb, keep = self._pair(force)
        lib().orc_set_force(self._h, m, a, b, pa, pb)

    def set_force_rate(self, rate):
        """dF/dt (None, (dfx, dfy) or fields) used by the next steps."""
        m, a, b, pa, pb, keep = self._pair(rate)
        lib().orc_set_force_rate(self._h, m, a, b, pa, pb)

    def init_rho0(self, rho):
        """alpha = 0 state feq_{j,0}(rho0, u) with u of the current state."""
        a = np.ascontiguousarray(rho, dtype=np.float64).ravel()
        assert a.size == self.nx * self.ny
        if lib().orc_init_rho0(self._h, _ptr(a)) != 0:
            raise ValueError("this oracle does not evolve rho0")

    def rho0(self):
        out = np.empty((self.ny, self.nx))
        if lib().orc_rho0(self._h, _ptr(out)) != 0:
            raise ValueError("this oracle does not evolve rho0")
        return out

    def rho0_state(self):
        out = np.empty((5, self.ny, self.nx))
        if lib().orc_get_rho0_state(self._h, _ptr(out)) != 0:
            raise ValueError("this oracle does not evolve rho0")
        return out

    def set_rho0_state(self, r):
        a = np.ascontiguousarray(r, dtype=np.float64)
        assert a.shape == (5, self.ny, self.nx)
        if lib().orc_set_rho0_state(self._h, _ptr(a)) != 0:
            raise ValueError("this oracle does not evolve rho0")

    def set_source(self, R):
        """Source R of the continuity equation (None, a constant or a field)."""
        if R is None:
            st = lib().orc_set_source(self._h, 0, 0.0, None)
        elif np.isscalar(R):
            st = lib().orc_set_source(self._h, 1, float(R), None)
        else:
            a = np.ascontiguousarray(R, dtype=np.float64).ravel()
            st = lib().orc_set_source(self._h, 2, 0.0, _ptr(a))
        if st != 0:
            raise ValueError("the source term needs a Newtonian fluid")

    def set_metrics(self, xi_x, xi_y, eta_x, eta_y):
        """Metric coefficients of a curvilinear grid given by the caller (ny x nx
        each) in place of those differenced from the node coordinates."""
        a = [np.ascontiguousarray(m, dtype=np.float64).ravel() for m in (xi_x, xi_y, eta_x, eta_y)]
        if any(m.size != self.nx * self.ny for m in a):
            raise ValueError("metric arrays must have ny x nx entries")
        if lib().orc_set_metrics(self._h, *(_ptr(m) for m in a)) != 0:
            raise ValueError("given metrics need a curvilinear grid")

    def metrics(self):
        """The metric coefficients xi_x, xi_y, eta_x, eta_y (ny x nx each) the
        step uses on a curvilinear grid."""
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        if lib().orc_get_metrics(self._h, *(_ptr(m) for m in out)) != 0:
            raise ValueError("metrics exist only on a curvilinear grid")
        return tuple(out)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    @property
    def dt(self):
        return lib().orc_dt(self._h)

    @property
    def cs2(self):
        return lib().orc_cs2(self._h)

    @property
    def steps(self):
        return lib().orc_steps(self._h)

    def init(self, u, v, p):
        a = [np.ascontiguousarray(t, dtype=np.float64) for t in (u, v, p)]
        lib().orc_init(self._h, *[_ptr(t) for t in a])

    def set_state(self, fh):
        fh = np.ascontiguousarray(fh, dtype=np.float64)
        assert fh.shape == (2, 5, self.ny, self.nx)
        lib().orc_set_state(self._h, _ptr(fh))

    def state(self):
        out = np.empty((2, 5, self.ny, self.nx), dtype=np.float64)
        lib().orc_get_state(self._h, _ptr(out))
        return out

    def step(self, n=1):
        lib().orc_step(self._h, int(n))

    def fields(self):
        out = np.empty((len(FIELD_NAMES), self.ny, self.nx), dtype=np.float64)
        lib().orc_fields(self._h, _ptr(out))
        return dict(zip(FIELD_NAMES, out))

    def collision_matrix(self, s):
        out = np.empty((5, 5), dtype=np.float64)
        lib().orc_collision_matrix(self._h, float(s), _ptr(out))
        return out

    def lambda_matrix(self):
        out = np.empty((5, 5), dtype=np.float64)
        lib().orc_lambda_matrix(self._h, _ptr(out))
        return out


def max_threads():
    return lib().orc_max_threads()
