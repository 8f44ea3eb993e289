"""FP64 CPU oracle for the lattice Boltzmann step of arXiv:1505.03271.

TEST INFRASTRUCTURE ONLY.  This package wraps ``lbref.c`` (plain C, FP64,
one cell at a time) with ctypes.  Only the test suite, the smoke check and
the benchmark's CPU-baseline leg may import it; the CUDA library never does,
and this package never imports the CUDA library.

Functions with a pin in ``tests/test_oracle_*.py``: lattice constants,
face generators, Lagrange/QUICK weights, equilibrium, Guo force, the ST step,
the FV step, the wall rules (the isothermal plates through the exactly
steady conduction state) and the observables.

The force part of the FV advected field is (dt/2)(1 - dt/(2 tau~)) F, the
plain population of Appendix A's inversion; its pin is the hydrostatic
column that stays at rest (tests/test_oracle_steps.py).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbref.c")
_SRCS = [_SRC, os.path.join(_HERE, "lbref3.c")]
_LIB = os.path.join(_HERE, "liblbref.so")

UNIFORM, TANH, SINH, CHEB = 0, 1, 2, 3
PERIODIC, WALLS, DENSITY = 0, 1, 2
INIT_TGV, INIT_SHEAR, INIT_POISEUILLE, INIT_RB = 0, 1, 2, 3
FV_HEUN, FV_SEMI, FV_EULER = 0, 1, 2
Q = 9


def build(force: bool = False) -> str:
    """Compile ``liblbref.so`` with gcc (IEEE FP64, no FMA contraction)."""
    deps = _SRCS + [os.path.join(_HERE, n) for n in ("lbref.h", "lbref3.h")]
    if not force and os.path.exists(_LIB) and all(os.path.getmtime(_LIB) >= os.path.getmtime(d) for d in deps):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", *_SRCS, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB)
    return _LIB


class Desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("lx", C.c_double), ("ly", C.c_double),
                ("sx", C.c_int), ("sy", C.c_int), ("stretch_x", C.c_double),
                ("stretch_y", C.c_double), ("bcx", C.c_int), ("bcy", C.c_int),
                ("thermal", C.c_int)]


class Params(C.Structure):
    _fields_ = [("tau", C.c_double), ("dt", C.c_double), ("tau_g", C.c_double),
                ("ax", C.c_double), ("ay", C.c_double), ("beta", C.c_double),
                ("grav", C.c_double), ("T0", C.c_double), ("T_bot", C.c_double),
                ("T_top", C.c_double)]


class Desc3(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("lx", C.c_double),
                ("ly", C.c_double), ("lz", C.c_double), ("sx", C.c_int), ("sy", C.c_int),
                ("sz", C.c_int), ("stretch_x", C.c_double), ("stretch_y", C.c_double),
                ("stretch_z", C.c_double), ("bcx", C.c_int), ("bcy", C.c_int), ("bcz", C.c_int),
                ("thermal", C.c_int)]


class Params3(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("tau", "dt", "tau_g", "ax", "ay", "az", "beta", "grav",
                                          "T0", "T_bot", "T_top")]


_lib = None
_D = C.POINTER(C.c_double)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.ref_create.restype = C.c_void_p
        L.ref_create.argtypes = [C.POINTER(Desc)]
        L.ref_destroy.argtypes = [C.c_void_p]
        L.ref_set_params.argtypes = [C.c_void_p, C.POINTER(Params)]
        L.ref_set_threads.argtypes = [C.c_int]
        L.ref_get_threads.restype = C.c_int
        L.ref_centers.argtypes = [C.c_void_p, _D, _D]
        L.ref_face_coords.argtypes = [C.c_void_p, _D, _D]
        L.ref_init_fields.argtypes = [C.c_void_p, _D, _D, _D, _D]
        L.ref_init_preset.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int,
                                      C.c_ulonglong]
        L.ref_set_pops.argtypes = [C.c_void_p, _D, _D]
        L.ref_get_pops.argtypes = [C.c_void_p, _D, _D]
        L.ref_step_st.argtypes = [C.c_void_p, C.c_int]
        L.ref_step_fv.argtypes = [C.c_void_p, C.c_int]
        L.ref_set_scheme.argtypes = [C.c_void_p, C.c_int]
        L.ref_set_boundary_density.argtypes = [C.c_void_p] + [C.c_double] * 4
        L.ref_moments.argtypes = [C.c_void_p, _D, _D, _D, _D]
        L.ref_conservation.argtypes = [C.c_void_p, _D, _D, _D, _D]
        L.ref_nusselt.argtypes = [C.c_void_p, _D, _D, _D]
        L.ref_lattice.argtypes = [C.POINTER(C.c_int), C.POINTER(C.c_int), _D, C.POINTER(C.c_int)]
        L.ref_faces.argtypes = [C.c_int, C.c_double, C.c_int, C.c_double, _D]
        L.ref_lagrange3.argtypes = [_D, C.c_double, _D]
        L.ref_equilibrium.argtypes = [C.c_double, C.c_double, C.c_double, _D]
        L.ref_guo_force.argtypes = [C.c_double] * 5 + [_D]
        L.ref_splitmix_uniform.restype = C.c_double
        L.ref_splitmix_uniform.argtypes = [C.c_ulonglong, C.c_ulonglong]
        L.ref3_create.restype = C.c_void_p
        L.ref3_create.argtypes = [C.POINTER(Desc3)]
        L.ref3_destroy.argtypes = [C.c_void_p]
        L.ref3_set_params.argtypes = [C.c_void_p, C.POINTER(Params3)]
        L.ref3_init_preset.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_int,
                                       C.c_ulonglong]
        L.ref3_init_fields.argtypes = [C.c_void_p] + [_D] * 5
        L.ref3_set_pops.argtypes = [C.c_void_p, _D, _D]
        L.ref3_get_pops.argtypes = [C.c_void_p, _D, _D]
        L.ref3_step_st.argtypes = [C.c_void_p, C.c_int]
        L.ref3_step_fv.argtypes = [C.c_void_p, C.c_int]
        L.ref3_moments.argtypes = [C.c_void_p] + [_D] * 5
        L.ref3_conservation.argtypes = [C.c_void_p] + [_D] * 5
        L.ref3_nusselt.argtypes = [C.c_void_p, _D, _D, _D]
        L.ref3_lattice.argtypes = [C.POINTER(C.c_int)] * 3 + [_D, C.POINTER(C.c_int)]
        L.ref3_equilibrium.argtypes = [C.c_double] * 4 + [_D]
        L.ref3_guo_force.argtypes = [C.c_double] * 7 + [_D]
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _c64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    lib().ref_set_threads(int(n))


def get_threads() -> int:
    return int(lib().ref_get_threads())


def lattice():
    cx = (C.c_int * Q)()
    cy = (C.c_int * Q)()
    w = (C.c_double * Q)()
    inv = (C.c_int * Q)()
    lib().ref_lattice(cx, cy, w, inv)
    return (np.array(cx[:]), np.array(cy[:]), np.array(w[:]), np.array(inv[:]))


def faces(n, L, spacing=UNIFORM, stretch=0.0):
    xi = np.zeros(n + 1)
    lib().ref_faces(int(n), float(L), int(spacing), float(stretch), _p(xi))
    return xi


def lagrange3(pos, x):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    w = np.zeros(3)
    lib().ref_lagrange3(_p(pos), float(x), _p(w))
    return w


def equilibrium(rho, ux, uy):
    out = np.zeros(Q)
    lib().ref_equilibrium(float(rho), float(ux), float(uy), _p(out))
    return out


def guo_force(rho, ux, uy, ax, ay):
    out = np.zeros(Q)
    lib().ref_guo_force(float(rho), float(ux), float(uy), float(ax), float(ay), _p(out))
    return out


def splitmix_uniform(seed, counter):
    return float(lib().ref_splitmix_uniform(int(seed), int(counter)))


class RefGrid:
    """One oracle grid: state f~ (and g~) as [9, ny, nx] FP64 arrays."""

    def __init__(self, nx, ny, lx=None, ly=None, sx=UNIFORM, sy=UNIFORM, stretch_x=0.0,
                 stretch_y=0.0, bcx=PERIODIC, bcy=PERIODIC, thermal=False):
        self.desc = Desc(int(nx), int(ny), float(lx if lx is not None else nx),
                         float(ly if ly is not None else ny), int(sx), int(sy),
                         float(stretch_x), float(stretch_y), int(bcx), int(bcy), int(bool(thermal)))
        self.nx, self.ny, self.thermal = int(nx), int(ny), bool(thermal)
        h = lib().ref_create(C.byref(self.desc))
        if not h:
            raise ValueError("oracle rejected the grid description")
        self._h = C.c_void_p(h)

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.ref_destroy(self._h)
            self._h = None

    def set_params(self, tau, dt=1.0, tau_g=None, ax=0.0, ay=0.0, beta=0.0, grav=0.0, T0=1.0,
                   T_bot=1.0, T_top=1.0):
        self.params = Params(float(tau), float(dt), float(tau if tau_g is None else tau_g),
                             float(ax), float(ay), float(beta), float(grav), float(T0),
                             float(T_bot), float(T_top))
        if lib().ref_set_params(self._h, C.byref(self.params)) != 0:
            raise ValueError("oracle rejected the parameters")
        return self

    def centers(self):
        xc, yc = np.zeros(self.nx), np.zeros(self.ny)
        lib().ref_centers(self._h, _p(xc), _p(yc))
        return xc, yc

    def face_coords(self):
        a, b = np.zeros(self.nx + 1), np.zeros(self.ny + 1)
        lib().ref_face_coords(self._h, _p(a), _p(b))
        return a, b

    def init_fields(self, rho=None, ux=None, uy=None, T=None):
        arrs = [_c64(v) for v in (rho, ux, uy, T)]
        if lib().ref_init_fields(self._h, *[_p(a) for a in arrs]) != 0:
            raise ValueError("init_fields failed")
        return self

    def init_preset(self, kind, u0=0.0, amp=0.0, mode=1, seed=0):
        if lib().ref_init_preset(self._h, int(kind), float(u0), float(amp), int(mode),
                                 int(seed)) != 0:
            raise ValueError("init_preset failed")
        return self

    def set_pops(self, f, g=None):
        f = _c64(f)
        g = _c64(g)
        lib().ref_set_pops(self._h, _p(f), _p(g))
        return self

    def get_pops(self):
        f = np.zeros((Q, self.ny, self.nx))
        g = np.zeros((Q, self.ny, self.nx))
        lib().ref_get_pops(self._h, _p(f), _p(g))
        return (f, g) if self.thermal else (f, None)

    def step_st(self, n=1):
        if lib().ref_step_st(self._h, int(n)) != 0:
            raise ValueError("step_st rejected (needs uniform unit spacing and dt = 1)")
        return self

    def set_scheme(self, scheme):
        """FV_HEUN (Eq. (semi-heun)), FV_SEMI (Eq. (semi)) or FV_EULER
        (Eq. (euler), plain populations); call before initialising."""
        if lib().ref_set_scheme(self._h, int(scheme)) != 0:
            raise ValueError("unknown FV scheme %r" % (scheme,))
        return self

    def set_boundary_density(self, rho_x0=1.0, rho_x1=1.0, rho_y0=1.0, rho_y1=1.0):
        """Densities imposed on the faces of DENSITY axes (Sec. II B 5)."""
        if lib().ref_set_boundary_density(self._h, float(rho_x0), float(rho_x1), float(rho_y0),
                                          float(rho_y1)) != 0:
            raise ValueError("boundary densities must be > 0")
        return self

    def step_fv(self, n=1):
        if lib().ref_step_fv(self._h, int(n)) != 0:
            raise ValueError("step_fv failed")
        return self

    def moments(self):
        out = [np.zeros((self.ny, self.nx)) for _ in range(4)]
        lib().ref_moments(self._h, *[_p(a) for a in out])
        return tuple(out)

    def conservation(self):
        v = [C.c_double() for _ in range(4)]
        lib().ref_conservation(self._h, *[C.byref(x) for x in v])
        return tuple(x.value for x in v)

    def nusselt(self):
        v = [C.c_double() for _ in range(3)]
        if lib().ref_nusselt(self._h, *[C.byref(x) for x in v]) != 0:
            raise ValueError("nusselt needs a thermal grid")
        return tuple(x.value for x in v)


Q3 = 19


def lattice3():
    """D3Q19 velocities, weights and inverse map (cx, cy, cz, w, inv)."""
    cx, cy, cz, inv = [(C.c_int * Q3)() for _ in range(4)]
    w = np.zeros(Q3)
    lib().ref3_lattice(cx, cy, cz, _p(w), inv)
    return np.array(cx[:]), np.array(cy[:]), np.array(cz[:]), w, np.array(inv[:])


def equilibrium3(rho, ux, uy, uz):
    out = np.zeros(Q3)
    lib().ref3_equilibrium(float(rho), float(ux), float(uy), float(uz), _p(out))
    return out


def guo_force3(rho, ux, uy, uz, ax, ay, az):
    out = np.zeros(Q3)
    lib().ref3_guo_force(*[float(v) for v in (rho, ux, uy, uz, ax, ay, az)], _p(out))
    return out


class RefGrid3:
    """One D3Q19 oracle grid: state [19, nz, ny, nx] FP64 arrays; plates on z."""

    def __init__(self, nx, ny, nz, lx=None, ly=None, lz=None, sx=UNIFORM, sy=UNIFORM, sz=UNIFORM,
                 stretch_x=0.0, stretch_y=0.0, stretch_z=0.0, bcx=PERIODIC, bcy=PERIODIC, bcz=PERIODIC,
                 thermal=False):
        L = [float(v if v is not None else n) for v, n in ((lx, nx), (ly, ny), (lz, nz))]
        self.desc = Desc3(int(nx), int(ny), int(nz), *L, int(sx), int(sy), int(sz), float(stretch_x),
                          float(stretch_y), float(stretch_z), int(bcx), int(bcy), int(bcz),
                          int(bool(thermal)))
        self.shape = (int(nz), int(ny), int(nx))
        self.thermal = bool(thermal)
        h = lib().ref3_create(C.byref(self.desc))
        if not h:
            raise ValueError("oracle rejected the 3-D grid description")
        self._h = C.c_void_p(h)

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.ref3_destroy(self._h)
            self._h = None

    def set_params(self, tau, dt=1.0, tau_g=None, ax=0.0, ay=0.0, az=0.0, beta=0.0, grav=0.0, T0=1.0,
                   T_bot=1.0, T_top=1.0):
        self.params = Params3(float(tau), float(dt), float(tau if tau_g is None else tau_g), float(ax),
                              float(ay), float(az), float(beta), float(grav), float(T0), float(T_bot),
                              float(T_top))
        if lib().ref3_set_params(self._h, C.byref(self.params)) != 0:
            raise ValueError("oracle rejected the parameters")
        return self

    def init_preset(self, kind, u0=0.0, amp=0.0, mode=1, seed=0):
        if lib().ref3_init_preset(self._h, int(kind), float(u0), float(amp), int(mode), int(seed)) != 0:
            raise ValueError("init_preset failed")
        return self

    def init_fields(self, rho=None, ux=None, uy=None, uz=None, T=None):
        arrs = [_c64(v) for v in (rho, ux, uy, uz, T)]
        if lib().ref3_init_fields(self._h, *[_p(a) for a in arrs]) != 0:
            raise ValueError("init_fields failed")
        return self

    def set_pops(self, f, g=None):
        f, g = _c64(f), _c64(g)
        lib().ref3_set_pops(self._h, _p(f), _p(g))
        return self

    def get_pops(self):
        f = np.zeros((Q3,) + self.shape)
        g = np.zeros((Q3,) + self.shape)
        lib().ref3_get_pops(self._h, _p(f), _p(g))
        return (f, g) if self.thermal else (f, None)

    def step_st(self, n=1):
        if lib().ref3_step_st(self._h, int(n)) != 0:
            raise ValueError("step_st rejected (needs uniform unit spacing and dt = 1)")
        return self

    def step_fv(self, n=1):
        if lib().ref3_step_fv(self._h, int(n)) != 0:
            raise ValueError("step_fv failed")
        return self

    def moments(self):
        out = [np.zeros(self.shape) for _ in range(5)]
        lib().ref3_moments(self._h, *[_p(a) for a in out])
        return tuple(out)

    def conservation(self):
        v = [C.c_double() for _ in range(5)]
        lib().ref3_conservation(self._h, *[C.byref(x) for x in v])
        return tuple(x.value for x in v)

    def nusselt(self):
        v = [C.c_double() for _ in range(3)]
        if lib().ref3_nusselt(self._h, *[C.byref(x) for x in v]) != 0:
            raise ValueError("nusselt needs a thermal grid")
        return tuple(x.value for x in v)
