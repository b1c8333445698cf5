"""Python binding of the C ABI in include/lbm.h (ctypes; argument marshalling only).

Every function below has the name of the C entry point it wraps and forwards to it; all
arithmetic of the method runs in the CUDA library. If the library has not been built the
first call raises: there is no CPU fallback. ``Lattice`` is a small convenience wrapper that
owns one handle.

Arrays are numpy FP64, shaped (nz, ny, nx) for scalar fields, (3, nz, ny, nx) for vector
fields and (Q, nz, ny, nx) for populations.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

import numpy as np

LBM_D2Q9, LBM_D3Q19 = 9, 19
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_ENONFINITE, LBM_ETIMEOUT, LBM_ESTATE = 0, -1, -2, -3, -4, -5, -6
LBM_SCHEME_DIFFERENCE_FREE, LBM_SCHEME_FINITE_DIFFERENCE = 0, 1
LBM_STORAGE_FP32, LBM_STORAGE_FP16, LBM_STORAGE_BF16 = 0, 1, 2

_LIB_PATH = Path(__file__).resolve().parent / "_build" / "liblbm_gb300.so"
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class lbm_opts(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("storage", ctypes.c_int), ("courant", ctypes.c_double),
                ("walls", ctypes.c_int), ("stream", ctypes.c_void_p), ("graph_steps", ctypes.c_int)]


class LBMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"lbm status {status}: {message}")
        self.status = status


# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("lbm_default_opts", None, [ctypes.POINTER(lbm_opts)]),
    ("lbm_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), _ip, ctypes.c_int] + [ctypes.c_double] * 7
     + [_dp, ctypes.POINTER(lbm_opts)]),
    ("lbm_init_phi", ctypes.c_int, [ctypes.c_void_p, _dp, _dp, ctypes.c_double]),
    ("lbm_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("lbm_moments", ctypes.c_int, [ctypes.c_void_p, _dp, _dp, _dp]),
    ("lbm_gradients", ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    ("lbm_mass", ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    ("lbm_get_pops", ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    ("lbm_set_pops", ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    ("lbm_launch_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("lbm_tau_phi", ctypes.c_double, [ctypes.c_void_p]),
    ("lbm_lattice_tables", ctypes.c_int, [ctypes.c_int, _ip, _ip, _dp]),
    ("lbm_mass_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _ip, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    ("lbm_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("lbm_destroy", None, [ctypes.c_void_p]),
]

_lib = None


def library_path() -> Path:
    return _LIB_PATH


def load():
    """Load the CUDA library; raises if it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not _LIB_PATH.exists():
        raise RuntimeError(f"CUDA library {_LIB_PATH} is not built; run paper_2407_12263_gb300.build.build()")
    lib = ctypes.CDLL(str(_LIB_PATH))
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    if a.dtype != np.float64 or not a.flags.c_contiguous:
        raise TypeError("arrays must be C-contiguous float64")
    return a.ctypes.data_as(_dp)


def _check(h, status):
    if status != LBM_OK:
        msg = load().lbm_last_error(h)
        raise LBMError(status, msg.decode() if msg else "")
    return status


# ---------------------------------------------------------------- the C entry points
def lbm_default_opts() -> lbm_opts:
    o = lbm_opts()
    load().lbm_default_opts(ctypes.byref(o))
    return o


def lbm_create(grid, lattice, tau_f, tau_g, M, xi, sigma, rho_ratio=1.0, mu_ratio=1.0,
               body_force=(0.0, 0.0, 0.0), opts: lbm_opts | None = None):
    h = ctypes.c_void_p()
    g = (ctypes.c_int * 3)(*[int(v) for v in grid])
    bf = None if body_force is None else np.ascontiguousarray(body_force, dtype=np.float64)
    st = load().lbm_create(ctypes.byref(h), g, int(lattice), tau_f, tau_g, M, xi, sigma, rho_ratio, mu_ratio,
                           _ptr(bf), ctypes.byref(opts) if opts is not None else None)
    _check(None, st)
    return h


def lbm_init_phi(h, phi0, u0=None, p0=1.0 / 3.0):
    _check(h, load().lbm_init_phi(h, _ptr(phi0), _ptr(u0), p0))


def lbm_step(h, n):
    _check(h, load().lbm_step(h, int(n)))


def lbm_moments(h, phi=None, p=None, u=None):
    _check(h, load().lbm_moments(h, _ptr(phi), _ptr(p), _ptr(u)))


def lbm_gradients(h, grad_phi=None, normal=None):
    _check(h, load().lbm_gradients(h, _ptr(grad_phi), _ptr(normal)))


def lbm_mass(h):
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(h, load().lbm_mass(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def lbm_get_pops(h, f=None, g=None):
    _check(h, load().lbm_get_pops(h, _ptr(f), _ptr(g)))


def lbm_set_pops(h, f, g):
    _check(h, load().lbm_set_pops(h, _ptr(f), _ptr(g)))


def lbm_launch_count(h) -> int:
    return int(load().lbm_launch_count(h))


def lbm_tau_phi(h) -> float:
    return float(load().lbm_tau_phi(h))


def lbm_lattice_tables(lattice):
    d = ctypes.c_int()
    e = np.zeros(3 * lattice, dtype=np.int32)
    w = np.zeros(lattice)
    st = load().lbm_lattice_tables(int(lattice), ctypes.byref(d), e.ctypes.data_as(_ip), _ptr(w))
    if st != LBM_OK:
        raise LBMError(st, f"unknown lattice {lattice}")
    return d.value, e.reshape(lattice, 3).astype(np.int64), w


def lbm_mass_noalloc(g_device_ptr, lattice, grid, courant, rho_ratio, result_device_ptr, stream=None) -> int:
    """Mass sums of plain FP32 device populations into a caller-owned device triple, without
    any device allocation (raw device pointers in; returns the lbm status)."""
    gr = (ctypes.c_int * 3)(*[int(v) for v in grid])
    return int(load().lbm_mass_noalloc(ctypes.c_void_p(g_device_ptr), int(lattice), gr, courant, rho_ratio,
                                       ctypes.c_void_p(result_device_ptr), stream))


def lbm_last_error(h=None) -> str:
    return load().lbm_last_error(h).decode()


def lbm_destroy(h):
    if h:
        load().lbm_destroy(h)


# ---------------------------------------------------------------- convenience wrapper
class Lattice:
    """One handle; arrays shaped (nz, ny, nx). Same parameters as lbm_create."""

    def __init__(self, grid, lattice, tau_f, tau_g, M, xi, sigma, rho_ratio=1.0, mu_ratio=1.0,
                 body_force=(0.0, 0.0, 0.0), scheme=LBM_SCHEME_DIFFERENCE_FREE, courant=0.997, stream=None,
                 storage=LBM_STORAGE_FP32, graph_steps=None, walls=0):
        o = lbm_default_opts()
        o.scheme, o.courant, o.storage, o.walls = scheme, courant, storage, walls
        if graph_steps is not None:
            o.graph_steps = graph_steps
        o.stream = stream
        self.h = lbm_create(grid, lattice, tau_f, tau_g, M, xi, sigma, rho_ratio, mu_ratio, body_force, o)
        nx, ny, nz = grid
        self.Q, self.grid, self.shape, self.N = lattice, tuple(grid), (nz, ny, nx), nx * ny * nz

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def tau_phi(self):
        return lbm_tau_phi(self.h)

    @property
    def launch_count(self):
        return lbm_launch_count(self.h)

    def init_phi(self, phi0, u0=None, p0=1.0 / 3.0):
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(self.shape)
        u0 = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64).reshape((3,) + self.shape)
        lbm_init_phi(self.h, phi0, u0, p0)

    def step(self, n=1):
        lbm_step(self.h, n)

    def moments(self):
        phi, p, u = np.empty(self.shape), np.empty(self.shape), np.empty((3,) + self.shape)
        lbm_moments(self.h, phi, p, u)
        return phi, p, u

    def gradients(self):
        gphi, n = np.empty((3,) + self.shape), np.empty((3,) + self.shape)
        lbm_gradients(self.h, gphi, n)
        return gphi, n

    def mass(self):
        return lbm_mass(self.h)

    def get_pops(self):
        f, g = np.empty((self.Q,) + self.shape), np.empty((self.Q,) + self.shape)
        lbm_get_pops(self.h, f, g)
        return f, g

    def set_pops(self, f, g):
        lbm_set_pops(self.h, np.ascontiguousarray(f, dtype=np.float64), np.ascontiguousarray(g, dtype=np.float64))
