"""GB300 lattice Boltzmann library: FV (QUICK + semi-implicit + Heun) and ST
(collide-and-stream) time steps of arXiv:1505.03271 as CUDA kernels behind
the C ABI of ``include/lb.h``.

This module is the thin ctypes binding: it marshals arguments and raises
``LBError`` on a non-zero status.  Every step of the computation runs in the
CUDA library; there is no CPU path.  Loading fails loudly if the library
cannot be built or loaded.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _build

Q = 9

LB_OK, LB_ERR_ARG, LB_ERR_OOM, LB_ERR_CUDA, LB_ERR_STATE, LB_ERR_UNSTABLE, LB_ERR_TIMEOUT = range(7)
LB_AXIS_UNIFORM, LB_AXIS_TANH, LB_AXIS_SINH, LB_AXIS_CHEB = 0, 1, 2, 3
LB_BC_PERIODIC, LB_BC_WALLS, LB_BC_DENSITY = 0, 1, 2
LB_STORE_F64, LB_STORE_F32, LB_STORE_F16DEV, LB_STORE_BF16DEV = 0, 1, 2, 3
LB_INIT_TGV, LB_INIT_SHEAR, LB_INIT_POISEUILLE, LB_INIT_RB, LB_INIT_FIELDS = 0, 1, 2, 3, 4

STORE_NAMES = {"f64": LB_STORE_F64, "f32": LB_STORE_F32, "f16dev": LB_STORE_F16DEV,
               "bf16dev": LB_STORE_BF16DEV}
STORE_BYTES = {LB_STORE_F64: 8, LB_STORE_F32: 4, LB_STORE_F16DEV: 2, LB_STORE_BF16DEV: 2}


class LBError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"lb status {status}: {msg}")
        self.status = status


class lb_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("lx", C.c_double), ("ly", C.c_double),
                ("sx", C.c_int), ("sy", C.c_int), ("stretch_x", C.c_double),
                ("stretch_y", C.c_double), ("bcx", C.c_int), ("bcy", C.c_int),
                ("thermal", C.c_int), ("store", C.c_int), ("cuda_stream", C.c_void_p)]


class lb_params(C.Structure):
    _fields_ = [("tau", C.c_double), ("dt", C.c_double), ("tau_g", C.c_double),
                ("ax", C.c_double), ("ay", C.c_double), ("beta", C.c_double),
                ("grav", C.c_double), ("T0", C.c_double), ("T_bot", C.c_double),
                ("T_top", C.c_double)]


_DP = C.POINTER(C.c_double)


class lb_init_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("mode", C.c_int), ("u0", C.c_double), ("amp", C.c_double),
                ("seed", C.c_ulonglong), ("rho", _DP), ("ux", _DP), ("uy", _DP), ("T", _DP)]


class lb3_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("lx", C.c_double),
                ("ly", C.c_double), ("lz", C.c_double), ("sx", C.c_int), ("sy", C.c_int),
                ("sz", C.c_int), ("stretch_x", C.c_double), ("stretch_y", C.c_double),
                ("stretch_z", C.c_double), ("bcx", C.c_int), ("bcy", C.c_int), ("bcz", C.c_int),
                ("thermal", C.c_int), ("store", C.c_int), ("cuda_stream", C.c_void_p)]


class lb3_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("tau", "dt", "tau_g", "ax", "ay", "az", "beta", "grav",
                                          "T0", "T_bot", "T_top")]


class lb3_init_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("mode", C.c_int), ("u0", C.c_double), ("amp", C.c_double),
                ("seed", C.c_ulonglong), ("rho", _DP), ("ux", _DP), ("uy", _DP), ("uz", _DP),
                ("T", _DP)]


class lb_request(C.Structure):
    _fields_ = [("id", C.c_longlong), ("grid", lb_grid_desc), ("params", lb_params),
                ("init", lb_init_desc), ("nsteps", C.c_int)]


class lb_result(C.Structure):
    _fields_ = [("id", C.c_longlong), ("status", C.c_int), ("steps", C.c_int), ("cells", C.c_longlong),
                ("nu_vol", C.c_double), ("nu_bot", C.c_double), ("nu_top", C.c_double),
                ("mass", C.c_double), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double)]


SYMBOLS = ["lb_create_grid", "lb_init", "lb_step_fv", "lb_step_st", "lb_moments",
           "lb_conservation", "lb_nusselt", "lb_set_populations", "lb_get_populations",
           "lb_get_window", "lb_sync", "lb_destroy", "lb_last_error", "lb_kernel_launches",
           "lb_conservation_noalloc", "lb_set_fv_schedule", "lb_get_fv_schedule",
           "lb_set_fv_scheme", "lb_get_fv_scheme", "lb_set_boundary_density",
           "lb_set_graph_steps", "lb_get_graph_steps",
           "lb3_create_grid", "lb3_init", "lb3_step_fv", "lb3_step_st", "lb3_moments",
           "lb3_conservation", "lb3_nusselt", "lb3_set_populations", "lb3_get_populations", "lb3_sync",
           "lb3_destroy", "lb3_set_fv_schedule", "lb3_get_fv_schedule", "lb3_debug_drop_copies",
           "lb3_set_fv_staged_shape", "lb3_get_fv_staged_shape", "lb3_autotune_fv",
           "lb_autotune_fv", "lb_server_create", "lb_server_submit", "lb_server_pump",
           "lb_server_results", "lb_server_clock", "lb_server_destroy"]
LB_FV_AUTO, LB_FV_TILE, LB_FV_MARCH, LB_FV_PAIR, LB_FV_PTILE, LB_FV_SPLIT = 0, 1, 2, 3, 4, 5
LB_SERVE_SHARE, LB_SERVE_SHORTEST, LB_SERVE_ARRIVAL = 0, 1, 2
LB_FV_HEUN, LB_FV_SEMI, LB_FV_EULER = 0, 1, 2
LB3_FV_AUTO, LB3_FV_PLAIN, LB3_FV_STAGED = 0, 1, 2

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build: bool = True) -> C.CDLL:
    """Load (building first if it is stale) the CUDA library."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"CUDA library missing: {_build.LIB} (run __graft_entry__.build())")
    L = C.CDLL(_build.LIB)
    G = C.c_void_p
    L.lb_create_grid.argtypes = [C.POINTER(lb_grid_desc), C.POINTER(G)]
    L.lb_init.argtypes = [G, C.POINTER(lb_params), C.POINTER(lb_init_desc)]
    L.lb_step_fv.argtypes = [G, C.c_int]
    L.lb_step_st.argtypes = [G, C.c_int]
    L.lb_moments.argtypes = [G, _DP, _DP, _DP, _DP]
    L.lb_conservation.argtypes = [G, _DP, _DP, _DP, _DP]
    L.lb_nusselt.argtypes = [G, _DP, _DP, _DP]
    L.lb_set_populations.argtypes = [G, _DP, _DP]
    L.lb_get_populations.argtypes = [G, _DP, _DP]
    L.lb_get_window.argtypes = [G, C.c_int, C.c_int, C.c_int, C.c_int, _DP, _DP]
    L.lb_conservation_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                          C.c_void_p, C.c_void_p] + [C.c_double] * 5 + [
                                          C.c_void_p, C.c_void_p]
    L.lb_set_fv_schedule.argtypes = [G, C.c_int, C.c_int]
    L.lb_get_fv_schedule.argtypes = [G, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.lb_autotune_fv.argtypes = [G, C.c_int]
    L.lb_set_fv_scheme.argtypes = [G, C.c_int]
    L.lb_set_boundary_density.argtypes = [G] + [C.c_double] * 4
    L.lb_get_fv_scheme.argtypes = [G, C.POINTER(C.c_int)]
    L.lb_set_graph_steps.argtypes = [G, C.c_int]
    L.lb_get_graph_steps.argtypes = [G, C.POINTER(C.c_int), C.POINTER(C.c_ulonglong)]
    L.lb_server_create.argtypes = [C.c_int, C.c_int, C.c_ulonglong, C.c_int, C.c_int, C.c_void_p,
                                   C.POINTER(C.c_void_p)]
    L.lb_server_submit.argtypes = [C.c_void_p, C.POINTER(lb_request)]
    L.lb_server_pump.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.lb_server_results.argtypes = [C.c_void_p, C.POINTER(lb_result), C.c_int, C.POINTER(C.c_int)]
    L.lb_server_clock.argtypes = [C.c_void_p]
    L.lb_server_clock.restype = C.c_double
    L.lb_server_destroy.argtypes = [C.c_void_p]
    L.lb3_create_grid.argtypes = [C.POINTER(lb3_grid_desc), C.POINTER(G)]
    L.lb3_init.argtypes = [G, C.POINTER(lb3_params), C.POINTER(lb3_init_desc)]
    L.lb3_step_fv.argtypes = [G, C.c_int]
    L.lb3_step_st.argtypes = [G, C.c_int]
    L.lb3_moments.argtypes = [G] + [_DP] * 5
    L.lb3_conservation.argtypes = [G] + [_DP] * 5
    L.lb3_nusselt.argtypes = [G, _DP, _DP, _DP]
    L.lb3_set_populations.argtypes = [G, _DP, _DP]
    L.lb3_get_populations.argtypes = [G, _DP, _DP]
    L.lb3_sync.argtypes = [G]
    L.lb3_set_fv_schedule.argtypes = [G, C.c_int]
    L.lb3_get_fv_schedule.argtypes = [G, C.POINTER(C.c_int)]
    L.lb3_debug_drop_copies.argtypes = [G, C.c_int]
    L.lb3_set_fv_staged_shape.argtypes = [G, C.c_int, C.c_int, C.c_int]
    L.lb3_get_fv_staged_shape.argtypes = [G] + [C.POINTER(C.c_int)] * 3
    L.lb3_autotune_fv.argtypes = [G, C.c_int]
    L.lb3_destroy.argtypes = [G]
    L.lb_sync.argtypes = [G]
    L.lb_destroy.argtypes = [G]
    L.lb_last_error.restype = C.c_char_p
    L.lb_kernel_launches.restype = C.c_ulonglong
    for name in SYMBOLS:
        if name not in ("lb_last_error", "lb_kernel_launches", "lb_server_clock"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _check(status: int) -> None:
    if status != LB_OK:
        raise LBError(status, _lib.lb_last_error().decode())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_DP)


def _c64(a, shape=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------- C names --

def lb_create_grid(desc: lb_grid_desc) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().lb_create_grid(C.byref(desc), C.byref(h)))
    return h


def lb_init(grid, params: lb_params, init: lb_init_desc) -> None:
    _check(load().lb_init(grid, C.byref(params), C.byref(init)))


def lb_step_fv(grid, nsteps: int) -> None:
    _check(load().lb_step_fv(grid, int(nsteps)))


def lb_step_st(grid, nsteps: int) -> None:
    _check(load().lb_step_st(grid, int(nsteps)))


def lb_moments(grid, rho, ux, uy, T) -> None:
    _check(load().lb_moments(grid, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(T)))


def lb_conservation(grid):
    v = [C.c_double() for _ in range(4)]
    _check(load().lb_conservation(grid, *[C.byref(x) for x in v]))
    return tuple(x.value for x in v)


def lb_nusselt(grid):
    v = [C.c_double() for _ in range(3)]
    _check(load().lb_nusselt(grid, *[C.byref(x) for x in v]))
    return tuple(x.value for x in v)


def lb_set_populations(grid, f, g) -> None:
    _check(load().lb_set_populations(grid, _ptr(f), _ptr(g)))


def lb_get_populations(grid, f, g) -> None:
    _check(load().lb_get_populations(grid, _ptr(f), _ptr(g)))


def lb_get_window(grid, x0, y0, w, h, f, g) -> None:
    _check(load().lb_get_window(grid, int(x0), int(y0), int(w), int(h), _ptr(f), _ptr(g)))


def lb_conservation_noalloc(f_ptr, g_ptr, nx, ny, pitch, dx_ptr, dy_ptr, dt, ax, ay, beta_grav,
                            T0, out_ptr, stream=None) -> None:
    """Conservation sums of caller-owned device buffers (raw device addresses
    as ints), without any allocation; `out_ptr` receives 4 doubles on
    `stream`.  See include/lb.h for the limits."""
    _check(load().lb_conservation_noalloc(f_ptr, g_ptr, int(nx), int(ny), int(pitch), dx_ptr,
                                          dy_ptr, float(dt), float(ax), float(ay),
                                          float(beta_grav), float(T0), out_ptr, stream))


def lb_set_fv_schedule(grid, kernel: int, chunk: int = 0) -> None:
    _check(load().lb_set_fv_schedule(grid, int(kernel), int(chunk)))


def lb_set_fv_scheme(grid, scheme: int) -> None:
    _check(load().lb_set_fv_scheme(grid, int(scheme)))


def lb_set_boundary_density(grid, rho_x0=1.0, rho_x1=1.0, rho_y0=1.0, rho_y1=1.0) -> None:
    _check(load().lb_set_boundary_density(grid, float(rho_x0), float(rho_x1), float(rho_y0), float(rho_y1)))


def lb_get_fv_scheme(grid) -> int:
    v = C.c_int()
    _check(load().lb_get_fv_scheme(grid, C.byref(v)))
    return v.value


def lb_get_fv_schedule(grid):
    k, c = C.c_int(), C.c_int()
    _check(load().lb_get_fv_schedule(grid, C.byref(k), C.byref(c)))
    return k.value, c.value


def lb_set_graph_steps(grid, n: int) -> None:
    _check(load().lb_set_graph_steps(grid, int(n)))


def lb_get_graph_steps(grid):
    n, r = C.c_int(), C.c_ulonglong()
    _check(load().lb_get_graph_steps(grid, C.byref(n), C.byref(r)))
    return n.value, r.value


def lb_autotune_fv(grid, steps: int = 5) -> None:
    _check(load().lb_autotune_fv(grid, int(steps)))


def lb_sync(grid) -> None:
    _check(load().lb_sync(grid))


def lb_destroy(grid) -> None:
    _check(load().lb_destroy(grid))


def lb_last_error() -> str:
    return load().lb_last_error().decode()


def lb_kernel_launches() -> int:
    return int(load().lb_kernel_launches())


# ------------------------------------------------------- convenience class --

def current_stream_handle():
    """Handle of torch's current CUDA stream (PyTorch provides the streams)."""
    import torch
    return torch.cuda.current_stream().cuda_stream


class Grid:
    """A grid on the GPU.  Arrays returned are host numpy FP64 [ny, nx]."""

    def __init__(self, nx, ny, lx=None, ly=None, sx=LB_AXIS_UNIFORM, sy=LB_AXIS_UNIFORM,
                 stretch_x=0.0, stretch_y=0.0, bcx=LB_BC_PERIODIC, bcy=LB_BC_PERIODIC,
                 thermal=False, store=LB_STORE_F32, stream=None):
        if isinstance(store, str):
            store = STORE_NAMES[store]
        if stream is None:
            stream = current_stream_handle()
        self.desc = lb_grid_desc(int(nx), int(ny), float(nx if lx is None else lx),
                                 float(ny if ly is None else ly), int(sx), int(sy),
                                 float(stretch_x), float(stretch_y), int(bcx), int(bcy),
                                 int(bool(thermal)), int(store), C.c_void_p(stream or 0))
        self.nx, self.ny, self.thermal, self.store = int(nx), int(ny), bool(thermal), int(store)
        self._h = lb_create_grid(self.desc)

    def close(self):
        if getattr(self, "_h", None) is not None:
            lb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def init(self, tau, dt=1.0, tau_g=None, ax=0.0, ay=0.0, beta=0.0, grav=0.0, T0=1.0, T_bot=1.0,
             T_top=1.0, kind=LB_INIT_FIELDS, u0=0.0, amp=0.0, mode=1, seed=0, rho=None, ux=None,
             uy=None, T=None):
        self.params = lb_params(float(tau), float(dt), float(tau if tau_g is None else tau_g),
                                float(ax), float(ay), float(beta), float(grav), float(T0),
                                float(T_bot), float(T_top))
        shp = (self.ny, self.nx)
        keep = [_c64(v, shp) for v in (rho, ux, uy, T)]
        d = lb_init_desc(int(kind), int(mode), float(u0), float(amp), int(seed),
                         *[_ptr(a) for a in keep])
        lb_init(self._h, self.params, d)
        return self

    def step_fv(self, n=1):
        lb_step_fv(self._h, n)
        return self

    def step_st(self, n=1):
        lb_step_st(self._h, n)
        return self

    def moments(self):
        out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        lb_moments(self._h, *out)
        return tuple(out)

    def conservation(self):
        return lb_conservation(self._h)

    def nusselt(self):
        return lb_nusselt(self._h)

    def set_pops(self, f, g=None):
        shp = (Q, self.ny, self.nx)
        f, g = _c64(f, shp), _c64(g, shp)
        lb_set_populations(self._h, f, g)
        return self

    def get_pops(self):
        f = np.empty((Q, self.ny, self.nx))
        g = np.empty((Q, self.ny, self.nx)) if self.thermal else None
        lb_get_populations(self._h, f, g)
        return f, g

    def get_window(self, x0, y0, w, h):
        f = np.empty((Q, h, w))
        g = np.empty((Q, h, w)) if self.thermal else None
        lb_get_window(self._h, x0, y0, w, h, f, g)
        return f, g

    def set_fv_schedule(self, kernel, chunk=0):
        lb_set_fv_schedule(self._h, kernel, chunk)
        return self

    def fv_schedule(self):
        return lb_get_fv_schedule(self._h)

    def set_graph_steps(self, n):
        """Steps per replayed CUDA graph of long step runs (even; 0: off)."""
        lb_set_graph_steps(self._h, n)
        return self

    def graph_steps(self):
        """(graph length, graph replays issued so far)."""
        return lb_get_graph_steps(self._h)

    def set_fv_scheme(self, scheme):
        """LB_FV_HEUN, LB_FV_SEMI or LB_FV_EULER; a change needs init() again."""
        lb_set_fv_scheme(self._h, scheme)
        return self

    def fv_scheme(self):
        return lb_get_fv_scheme(self._h)

    def set_boundary_density(self, rho_x0=1.0, rho_x1=1.0, rho_y0=1.0, rho_y1=1.0):
        """Densities on the faces of LB_BC_DENSITY axes (Sec. II B 5)."""
        lb_set_boundary_density(self._h, rho_x0, rho_x1, rho_y0, rho_y1)
        return self

    def autotune_fv(self, steps=5):
        lb_autotune_fv(self._h, steps)
        return self.fv_schedule()

    def sync(self):
        lb_sync(self._h)
        return self


class Server:
    """Continuous-batching server of FV requests (see include/lb.h)."""

    def __init__(self, store=LB_STORE_F32, thermal=True, hbm_budget=64 << 30, steps_per_launch=50,
                 policy=None, stream=None):
        if isinstance(store, str):
            store = STORE_NAMES[store]
        self.store, self.thermal = int(store), bool(thermal)
        h = C.c_void_p()
        policy = LB_SERVE_ARRIVAL if policy is None else int(policy)
        _check(load().lb_server_create(self.store, int(self.thermal), int(hbm_budget),
                                       int(steps_per_launch), policy, stream, C.byref(h)))
        self._h = h
        self._keep = {}

    def submit(self, rid, nsteps, nx, ny, lx=None, ly=None, sx=LB_AXIS_UNIFORM, sy=LB_AXIS_UNIFORM,
               stretch_x=0.0, stretch_y=0.0, bcx=LB_BC_PERIODIC, bcy=LB_BC_PERIODIC, tau=0.3, dt=1.0,
               tau_g=None, ax=0.0, ay=0.0, beta=0.0, grav=0.0, T0=1.0, T_bot=1.0, T_top=1.0,
               kind=LB_INIT_RB, u0=0.0, amp=0.0, mode=1, seed=0):
        req = lb_request()
        req.id = int(rid)
        req.grid = lb_grid_desc(int(nx), int(ny), float(nx if lx is None else lx),
                                float(ny if ly is None else ly), int(sx), int(sy), float(stretch_x),
                                float(stretch_y), int(bcx), int(bcy), int(self.thermal), self.store, None)
        req.params = lb_params(float(tau), float(dt), float(tau if tau_g is None else tau_g), float(ax),
                               float(ay), float(beta), float(grav), float(T0), float(T_bot), float(T_top))
        req.init = lb_init_desc(int(kind), int(mode), float(u0), float(amp), int(seed), None, None, None, None)
        req.nsteps = int(nsteps)
        _check(load().lb_server_submit(self._h, C.byref(req)))

    def pump(self):
        a, p = C.c_int(), C.c_int()
        _check(load().lb_server_pump(self._h, C.byref(a), C.byref(p)))
        return a.value, p.value

    def results(self, max_n=4096):
        buf = (lb_result * max_n)()
        n = C.c_int()
        _check(load().lb_server_results(self._h, buf, int(max_n), C.byref(n)))
        fields = [f for f, _ in lb_result._fields_]
        return [{f: getattr(buf[i], f) for f in fields} for i in range(n.value)]

    def clock(self):
        return float(load().lb_server_clock(self._h))

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().lb_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Grid3:
    """A D3Q19 grid on the GPU (include/lb3.h).  Arrays are host numpy FP64
    [nz, ny, nx]; populations [19, nz, ny, nx]."""

    def __init__(self, nx, ny, nz, lx=None, ly=None, lz=None, sx=LB_AXIS_UNIFORM, sy=LB_AXIS_UNIFORM,
                 sz=LB_AXIS_UNIFORM, stretch_x=0.0, stretch_y=0.0, stretch_z=0.0, bcx=LB_BC_PERIODIC,
                 bcy=LB_BC_PERIODIC, bcz=LB_BC_PERIODIC, thermal=False, store=LB_STORE_F32, stream=None):
        if isinstance(store, str):
            store = STORE_NAMES[store]
        if stream is None:
            stream = current_stream_handle()
        L = [float(n if v is None else v) for v, n in ((lx, nx), (ly, ny), (lz, nz))]
        self.desc = lb3_grid_desc(int(nx), int(ny), int(nz), *L, int(sx), int(sy), int(sz),
                                  float(stretch_x), float(stretch_y), float(stretch_z), int(bcx), int(bcy),
                                  int(bcz), int(bool(thermal)), int(store), C.c_void_p(stream or 0))
        self.shape = (int(nz), int(ny), int(nx))
        self.thermal, self.store = bool(thermal), int(store)
        h = C.c_void_p()
        _check(load().lb3_create_grid(C.byref(self.desc), C.byref(h)))
        self._h = h

    @property
    def cells(self):
        return self.shape[0] * self.shape[1] * self.shape[2]

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().lb3_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def init(self, tau, dt=1.0, tau_g=None, ax=0.0, ay=0.0, az=0.0, beta=0.0, grav=0.0, T0=1.0, T_bot=1.0,
             T_top=1.0, kind=LB_INIT_FIELDS, u0=0.0, amp=0.0, mode=1, seed=0, rho=None, ux=None, uy=None,
             uz=None, T=None):
        self.params = lb3_params(float(tau), float(dt), float(tau if tau_g is None else tau_g), float(ax),
                                 float(ay), float(az), float(beta), float(grav), float(T0), float(T_bot),
                                 float(T_top))
        keep = [_c64(v, self.shape) for v in (rho, ux, uy, uz, T)]
        d = lb3_init_desc(int(kind), int(mode), float(u0), float(amp), int(seed), *[_ptr(a) for a in keep])
        _check(load().lb3_init(self._h, C.byref(self.params), C.byref(d)))
        return self

    def step_fv(self, n=1):
        _check(load().lb3_step_fv(self._h, int(n)))
        return self

    def step_st(self, n=1):
        _check(load().lb3_step_st(self._h, int(n)))
        return self

    def moments(self):
        out = [np.zeros(self.shape) for _ in range(5)]
        _check(load().lb3_moments(self._h, *[_ptr(a) for a in out]))
        return tuple(out)

    def conservation(self):
        v = [C.c_double() for _ in range(5)]
        _check(load().lb3_conservation(self._h, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def nusselt(self):
        v = [C.c_double() for _ in range(3)]
        _check(load().lb3_nusselt(self._h, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def set_pops(self, f, g=None):
        f = _c64(f, (19,) + self.shape)
        g = _c64(g, (19,) + self.shape)
        _check(load().lb3_set_populations(self._h, _ptr(f), _ptr(g)))
        return self

    def get_pops(self):
        f = np.zeros((19,) + self.shape)
        g = np.zeros((19,) + self.shape) if self.thermal else None
        _check(load().lb3_get_populations(self._h, _ptr(f), _ptr(g)))
        return f, g

    def sync(self):
        _check(load().lb3_sync(self._h))
        return self

    def set_fv_schedule(self, schedule):
        """LB3_FV_AUTO, LB3_FV_PLAIN or LB3_FV_STAGED (flux passes of step_fv)."""
        _check(load().lb3_set_fv_schedule(self._h, int(schedule)))
        return self

    def set_staged_shape(self, rows=0, planes=0, ahead=0):
        """Rows per tile, z planes per CTA and planes in flight of the staged
        flux passes (0: default)."""
        _check(load().lb3_set_fv_staged_shape(self._h, int(rows), int(planes), int(ahead)))
        return self

    @property
    def staged_shape(self):
        """(rows per tile, planes per CTA, planes ahead) of the staged passes."""
        v = [C.c_int() for _ in range(3)]
        _check(load().lb3_get_fv_staged_shape(self._h, *[C.byref(x) for x in v]))
        return tuple(x.value for x in v)

    def autotune_fv(self, steps=3):
        """Time the flux schedules on the live state, keep the fastest (the
        state is restored)."""
        _check(load().lb3_autotune_fv(self._h, int(steps)))
        return self

    @property
    def fv_schedule(self):
        """The flux passes a step runs: LB3_FV_PLAIN or LB3_FV_STAGED."""
        v = C.c_int()
        _check(load().lb3_get_fv_schedule(self._h, C.byref(v)))
        return v.value

    def drop_copies(self, on=True):
        """Test hook of the staged passes' bounded waits (include/lb3.h)."""
        _check(load().lb3_debug_drop_copies(self._h, int(bool(on))))
        return self
