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
LBM_STORAGE_FP32, LBM_STORAGE_FP16, LBM_STORAGE_BF16, LBM_STORAGE_AUTO = 0, 1, 2, 3

_LIB_PATH = Path(__file__).resolve().parent / "_build" / "liblbm_gb300.so"
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class lbm_opts(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("storage", ctypes.c_int), ("courant", ctypes.c_double),
                ("walls", ctypes.c_int), ("stream", ctypes.c_void_p), ("graph_steps", ctypes.c_int)]


class lbm_case(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int * 3), ("lattice", ctypes.c_int), ("tau_f", ctypes.c_double),
                ("tau_g", ctypes.c_double), ("M", ctypes.c_double), ("xi", ctypes.c_double),
                ("sigma", ctypes.c_double), ("rho_ratio", ctypes.c_double), ("mu_ratio", ctypes.c_double),
                ("body_force", ctypes.c_double * 3), ("walls", ctypes.c_int), ("storage", ctypes.c_int),
                ("courant", ctypes.c_double)]


class lbm_batch_opts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("graph_steps", ctypes.c_int)]


class lbm_diag(ctypes.Structure):
    _fields_ = [("max_speed", ctypes.c_double), ("argmax", ctypes.c_longlong), ("kinetic", ctypes.c_double),
                ("p_in", ctypes.c_double), ("p_out", ctypes.c_double), ("n_in", ctypes.c_longlong),
                ("n_out", ctypes.c_longlong)]


class lbm_jump_report(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_int), ("mass_error", ctypes.c_double), ("relax_ratio", ctypes.c_double),
                ("interface_shift", ctypes.c_double), ("interface_limit", ctypes.c_double),
                ("seconds_surrogate", ctypes.c_double), ("projected", ctypes.c_int)]


class LBMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"lbm status {status}: {message}")
        self.status = status


# (name, restype, argtypes) of every exported entry point
SIGNATURES = [
    ("lbm_default_opts", None, [ctypes.POINTER(lbm_opts)]),
    ("lbm_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), _ip, ctypes.c_int] + [ctypes.c_double] * 7
     + [_dp, ctypes.POINTER(lbm_opts)]),
    ("lbm_state_bytes", ctypes.c_longlong, [ctypes.c_int, _ip, ctypes.c_int]),
    ("lbm_create_ext", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), _ip, ctypes.c_int] + [ctypes.c_double] * 7
     + [_dp, ctypes.POINTER(lbm_opts), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    ("lbm_init_phi", ctypes.c_int, [ctypes.c_void_p, _dp, _dp, ctypes.c_double]),
    ("lbm_init_fields", ctypes.c_int, [ctypes.c_void_p, _dp, _dp, _dp, ctypes.c_double]),
    ("lbm_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("lbm_graph_prepare", ctypes.c_int, [ctypes.c_void_p]),
    ("lbm_moments", ctypes.c_int, [ctypes.c_void_p, _dp, _dp, _dp]),
    ("lbm_gradients", ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    ("lbm_mass", ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    ("lbm_diagnostics", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                                       ctypes.c_double, ctypes.POINTER(lbm_diag)]),
    ("lbm_get_pops", ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    ("lbm_set_pops", ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    ("lbm_launch_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("lbm_tau_phi", ctypes.c_double, [ctypes.c_void_p]),
    ("lbm_lattice_tables", ctypes.c_int, [ctypes.c_int, _ip, _ip, _dp]),
    ("lbm_mass_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _ip, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]),
    ("lbm_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("lbm_destroy", None, [ctypes.c_void_p]),
    ("lbm_batch_default_opts", None, [ctypes.POINTER(lbm_batch_opts)]),
    ("lbm_batch_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.POINTER(lbm_case),
                                        ctypes.POINTER(lbm_batch_opts)]),
    ("lbm_batch_case", ctypes.c_void_p, [ctypes.c_void_p, ctypes.c_int]),
    ("lbm_batch_tune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("lbm_batch_case_config", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _ip, _ip, _ip]),
    ("lbm_batch_set_config", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, _ip, ctypes.c_int]),
    ("lbm_batch_step", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("lbm_batch_launch_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("lbm_batch_cells", ctypes.c_longlong, [ctypes.c_void_p]),
    ("lbm_batch_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("lbm_batch_destroy", None, [ctypes.c_void_p]),
    # include/lbm_surrogate.h
    ("lbm_net_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_ulonglong, ctypes.c_void_p]),
    ("lbm_net_param_count", ctypes.c_longlong, [ctypes.c_void_p]),
    ("lbm_net_get_params", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    ("lbm_net_set_params", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    ("lbm_net_get_grads", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    ("lbm_net_forward", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, _ip]),
    ("lbm_net_gradients", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, _ip, _dp]),
    ("lbm_net_set_loss_weights", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)]),
    ("lbm_net_adam", ctypes.c_int, [ctypes.c_void_p, ctypes.c_float]),
    ("lbm_net_fail_waits", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("lbm_net_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("lbm_net_destroy", None, [ctypes.c_void_p]),
    ("lbm_coarse_fields", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("lbm_coarse_phi", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    ("lbm_restart_from_coarse", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_double]),
    ("lbm_surrogate_jump", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                          ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.POINTER(lbm_jump_report)]),
    ("lbm_surrogate_reserve", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("lbm_project_workspace_bytes", ctypes.c_longlong, [_ip]),
    ("lbm_project_solenoidal", ctypes.c_int, [ctypes.c_void_p, _ip, ctypes.c_void_p, ctypes.c_longlong,
                                              ctypes.c_void_p]),
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


def lbm_state_bytes(lattice, grid, storage=LBM_STORAGE_FP32) -> int:
    g = (ctypes.c_int * 3)(*[int(v) for v in grid])
    return int(load().lbm_state_bytes(int(lattice), g, int(storage)))


def lbm_create_ext(grid, lattice, tau_f, tau_g, M, xi, sigma, rho_ratio=1.0, mu_ratio=1.0,
                   body_force=(0.0, 0.0, 0.0), opts: lbm_opts | None = None, fg0=0, fg1=0, bytes_each=0):
    """lbm_create on two caller-owned device buffers (raw device pointers)."""
    h = ctypes.c_void_p()
    g = (ctypes.c_int * 3)(*[int(v) for v in grid])
    bf = None if body_force is None else np.ascontiguousarray(body_force, dtype=np.float64)
    st = load().lbm_create_ext(ctypes.byref(h), g, int(lattice), tau_f, tau_g, M, xi, sigma, rho_ratio, mu_ratio,
                               _ptr(bf), ctypes.byref(opts) if opts is not None else None, ctypes.c_void_p(fg0),
                               ctypes.c_void_p(fg1), ctypes.c_size_t(int(bytes_each)))
    _check(None, st)
    return h


def lbm_init_phi(h, phi0, u0=None, p0=1.0 / 3.0):
    _check(h, load().lbm_init_phi(h, _ptr(phi0), _ptr(u0), p0))


def lbm_init_fields(h, phi0, u0=None, p=None, p0=1.0 / 3.0):
    _check(h, load().lbm_init_fields(h, _ptr(phi0), _ptr(u0), _ptr(p), p0))


def lbm_step(h, n):
    _check(h, load().lbm_step(h, int(n)))


def lbm_moments(h, phi=None, p=None, u=None):
    _check(h, load().lbm_moments(h, _ptr(phi), _ptr(p), _ptr(u)))


def lbm_gradients(h, grad_phi=None, normal=None):
    _check(h, load().lbm_gradients(h, _ptr(grad_phi), _ptr(normal)))


def lbm_diagnostics(h, centre, r_in, r_out):
    """Device-side diagnostics of the current state (see include/lbm.h): a dict with max_speed,
    argmax, kinetic, p_in, p_out, n_in, n_out."""
    c = (ctypes.c_double * 3)(*[float(v) for v in centre])
    d = lbm_diag()
    _check(h, load().lbm_diagnostics(h, c, float(r_in), float(r_out), ctypes.byref(d)))
    return {k: getattr(d, k) for k, _ in lbm_diag._fields_}


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


def lbm_mass_noalloc(g_device_ptr, lattice, grid, walls, courant, rho_ratio, result_device_ptr, stream=None) -> int:
    """Mass sums of plain FP32 device populations into a caller-owned device triple, without
    any device allocation (raw device pointers in; returns the lbm status)."""
    gr = (ctypes.c_int * 3)(*[int(v) for v in grid])
    return int(load().lbm_mass_noalloc(ctypes.c_void_p(g_device_ptr), int(lattice), gr, int(walls), courant,
                                       rho_ratio, ctypes.c_void_p(result_device_ptr), stream))


def lbm_last_error(h=None) -> str:
    return load().lbm_last_error(h).decode()


def lbm_destroy(h):
    if h:
        load().lbm_destroy(h)


def _bcheck(b, status):
    if status != LBM_OK:
        msg = load().lbm_batch_last_error(b)
        raise LBMError(status, msg.decode() if msg else "")
    return status


def lbm_batch_default_opts() -> lbm_batch_opts:
    o = lbm_batch_opts()
    load().lbm_batch_default_opts(ctypes.byref(o))
    return o


def make_case(grid, lattice, tau_f, tau_g, M, xi, sigma, rho_ratio=1.0, mu_ratio=1.0,
              body_force=(0.0, 0.0, 0.0), walls=0, storage=LBM_STORAGE_FP32, courant=0.0) -> lbm_case:
    c = lbm_case()
    c.grid[:] = [int(v) for v in grid]
    c.lattice, c.tau_f, c.tau_g, c.M, c.xi, c.sigma = int(lattice), tau_f, tau_g, M, xi, sigma
    c.rho_ratio, c.mu_ratio = rho_ratio, mu_ratio
    c.body_force[:] = [float(v) for v in body_force]
    c.walls, c.storage, c.courant = int(walls), int(storage), courant
    return c


def lbm_batch_create(cases, opts: lbm_batch_opts | None = None):
    arr = (lbm_case * len(cases))(*cases)
    b = ctypes.c_void_p()
    st = load().lbm_batch_create(ctypes.byref(b), len(cases), arr, ctypes.byref(opts) if opts is not None else None)
    _bcheck(None, st)
    return b


def lbm_batch_case(b, k):
    h = load().lbm_batch_case(b, int(k))
    if not h:
        raise LBMError(LBM_EINVAL, f"no case {k}")
    return ctypes.c_void_p(h)


def lbm_batch_tune(b, trial_steps):
    _bcheck(b, load().lbm_batch_tune(b, int(trial_steps)))


def lbm_batch_case_config(b, k):
    """(tile shape, storage, dedicated) of case k."""
    tile = (ctypes.c_int * 3)()
    storage, dedicated = ctypes.c_int(), ctypes.c_int()
    _bcheck(b, load().lbm_batch_case_config(b, int(k), tile, ctypes.byref(storage), ctypes.byref(dedicated)))
    return tuple(tile), storage.value, bool(dedicated.value)


def lbm_batch_set_config(b, k, tile=None, dedicated=False):
    t = None if tile is None else (ctypes.c_int * 3)(*[int(v) for v in tile])
    _bcheck(b, load().lbm_batch_set_config(b, int(k), t, int(bool(dedicated))))


def lbm_batch_step(b, n):
    _bcheck(b, load().lbm_batch_step(b, int(n)))


def lbm_batch_launch_count(b) -> int:
    return int(load().lbm_batch_launch_count(b))


def lbm_batch_cells(b) -> int:
    return int(load().lbm_batch_cells(b))


def lbm_batch_last_error(b=None) -> str:
    return load().lbm_batch_last_error(b).decode()


def lbm_batch_destroy(b):
    if b:
        load().lbm_batch_destroy(b)


# ---------------------------------------------------------------- convenience wrapper
class Lattice:
    """One handle; arrays shaped (nz, ny, nx). Same parameters as lbm_create."""

    def __init__(self, grid, lattice, tau_f=0.8, tau_g=0.8, M=0.02, xi=4.0, sigma=1e-3, rho_ratio=1.0, mu_ratio=1.0,
                 body_force=(0.0, 0.0, 0.0), scheme=LBM_SCHEME_DIFFERENCE_FREE, courant=0.997, stream=None,
                 storage=LBM_STORAGE_FP32, graph_steps=None, walls=0, handle=None, buffers=None):
        """buffers: None (the library allocates the state), or (fg0, fg1, bytes_each), two
        caller-owned device buffers (lbm_create_ext) that must outlive the handle."""
        if handle is not None:  # a handle owned elsewhere (a case of a Batch)
            self.h, self._owned = handle, False
            nx, ny, nz = grid
            self.Q, self.grid, self.shape, self.N = lattice, tuple(grid), (nz, ny, nx), nx * ny * nz
            return
        self._owned = True
        o = lbm_default_opts()
        o.scheme, o.courant, o.storage, o.walls = scheme, courant, storage, walls
        if graph_steps is not None:
            o.graph_steps = graph_steps
        o.stream = stream
        if buffers is None:
            self.h = lbm_create(grid, lattice, tau_f, tau_g, M, xi, sigma, rho_ratio, mu_ratio, body_force, o)
        else:
            fg0, fg1, nbytes = buffers
            self.h = lbm_create_ext(grid, lattice, tau_f, tau_g, M, xi, sigma, rho_ratio, mu_ratio, body_force, o,
                                    fg0, fg1, nbytes)
        nx, ny, nz = grid
        self.Q, self.grid, self.shape, self.N = lattice, tuple(grid), (nz, ny, nx), nx * ny * nz

    def close(self):
        if getattr(self, "h", None):
            if getattr(self, "_owned", True):
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

    def init_phi(self, phi0, u0=None, p0=1.0 / 3.0, p=None):
        """Initial state; p (a pressure field, optional) replaces the uniform p0 in f^eq."""
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(self.shape)
        u0 = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64).reshape((3,) + self.shape)
        if p is None:
            lbm_init_phi(self.h, phi0, u0, p0)
        else:
            lbm_init_fields(self.h, phi0, u0, np.ascontiguousarray(p, dtype=np.float64).reshape(self.shape), p0)

    def graph_prepare(self):
        """Capture and upload the step graph for the current buffer without running it."""
        _check(self.h, load().lbm_graph_prepare(self.h))

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

    def diagnostics(self, centre, r_in, r_out):
        return lbm_diagnostics(self.h, centre, r_in, r_out)

    def get_pops(self):
        f, g = np.empty((self.Q,) + self.shape), np.empty((self.Q,) + self.shape)
        lbm_get_pops(self.h, f, g)
        return f, g

    def set_pops(self, f, g):
        lbm_set_pops(self.h, np.ascontiguousarray(f, dtype=np.float64), np.ascontiguousarray(g, dtype=np.float64))


class Batch:
    """Many independent cases advanced by one launch per step. ``cases`` are lbm_case structs
    (see make_case); ``case(k)`` is a Lattice view of case k (owned by the batch)."""

    def __init__(self, cases, stream=None, graph_steps=None):
        o = lbm_batch_default_opts()
        o.stream = stream
        if graph_steps is not None:
            o.graph_steps = graph_steps
        self.b = lbm_batch_create(cases, o)
        self.n = len(cases)
        self._views = [Lattice(tuple(c.grid), c.lattice, handle=lbm_batch_case(self.b, k)) for k, c in enumerate(cases)]

    def close(self):
        if getattr(self, "b", None):
            for v in self._views:
                v.h = None
            lbm_batch_destroy(self.b)
            self.b = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def case(self, k) -> Lattice:
        return self._views[k]

    def tune(self, trial_steps=10):
        lbm_batch_tune(self.b, trial_steps)

    def config(self, k):
        """(tile, storage, dedicated) of case k."""
        return lbm_batch_case_config(self.b, k)

    def set_config(self, k, tile=None, dedicated=False):
        lbm_batch_set_config(self.b, k, tile, dedicated)

    def step(self, n=1):
        lbm_batch_step(self.b, n)

    @property
    def launch_count(self):
        return lbm_batch_launch_count(self.b)

    @property
    def cells(self):
        return lbm_batch_cells(self.b)


# ---------------------------------------------------------------- the surrogate (include/lbm_surrogate.h)
_fp = ctypes.POINTER(ctypes.c_float)


def _ncheck(n, status):
    if status != LBM_OK:
        msg = load().lbm_net_last_error(n)
        raise LBMError(status, msg.decode() if msg else "")
    return status


class Net:
    """The convolutional surrogate. Field batches are device FP32 arrays [B][5][D][H][W] passed
    by pointer (e.g. torch tensors' data_ptr()); grids are (nx, ny, nz). stream: the cudaStream_t
    handle the network runs on; None or 0 makes the library create a stream of its own, which is
    not ordered with torch's default stream (also handle 0), so pass a non-default stream that
    also runs the torch work producing the inputs."""

    def __init__(self, fp16=True, seed=0, stream=None):
        h = ctypes.c_void_p()
        _ncheck(None, load().lbm_net_create(ctypes.byref(h), int(bool(fp16)), int(seed), stream))
        self.n = h

    def close(self):
        if getattr(self, "n", None):
            load().lbm_net_destroy(self.n)
            self.n = None

    __del__ = close

    @property
    def param_count(self):
        return int(load().lbm_net_param_count(self.n))

    def get_params(self):
        a = np.empty(self.param_count, dtype=np.float32)
        _ncheck(self.n, load().lbm_net_get_params(self.n, a.ctypes.data_as(_fp)))
        return a

    def set_params(self, a):
        a = np.ascontiguousarray(a, dtype=np.float32)
        assert a.size == self.param_count
        _ncheck(self.n, load().lbm_net_set_params(self.n, a.ctypes.data_as(_fp)))

    def get_grads(self):
        a = np.empty(self.param_count, dtype=np.float32)
        _ncheck(self.n, load().lbm_net_get_grads(self.n, a.ctypes.data_as(_fp)))
        return a

    def forward(self, x_ptr, y_ptr, batch, grid):
        g = (ctypes.c_int * 3)(*[int(v) for v in grid])
        _ncheck(self.n, load().lbm_net_forward(self.n, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), int(batch), g))

    def gradients(self, x_ptr, t_ptr, batch, grid):
        g = (ctypes.c_int * 3)(*[int(v) for v in grid])
        loss = ctypes.c_double()
        _ncheck(self.n, load().lbm_net_gradients(self.n, ctypes.c_void_p(x_ptr), ctypes.c_void_p(t_ptr), int(batch), g,
                                                 ctypes.byref(loss)))
        return loss.value

    def set_loss_weights(self, w):
        a = (ctypes.c_float * 5)(*[float(v) for v in w])
        _ncheck(self.n, load().lbm_net_set_loss_weights(self.n, a))

    def adam(self, lr):
        _ncheck(self.n, load().lbm_net_adam(self.n, float(lr)))

    def fail_waits(self, on):
        _ncheck(self.n, load().lbm_net_fail_waits(self.n, int(bool(on))))


def lbm_coarse_fields(h, factor, out_ptr):
    _check(h, load().lbm_coarse_fields(h, int(factor), ctypes.c_void_p(out_ptr)))


def lbm_coarse_phi(h, factor, out_ptr):
    _check(h, load().lbm_coarse_phi(h, int(factor), ctypes.c_void_p(out_ptr)))


def lbm_restart_from_coarse(h, factor, coarse_ptr, p0=1.0 / 3.0):
    _check(h, load().lbm_restart_from_coarse(h, int(factor), ctypes.c_void_p(coarse_ptr), float(p0)))


def lbm_surrogate_reserve(h, factor):
    _check(h, load().lbm_surrogate_reserve(h, int(factor)))


def lbm_surrogate_jump(h, net, factor, mean_std, k, judge_steps, mass_tol, relax_tol, interface_tol=1.0):
    ms = (ctypes.c_float * 10)(*[float(v) for v in mean_std])
    rep = lbm_jump_report()
    _check(h, load().lbm_surrogate_jump(h, net.n, int(factor), ms, int(k), int(judge_steps), float(mass_tol),
                                        float(relax_tol), float(interface_tol), ctypes.byref(rep)))
    return {"accepted": bool(rep.accepted), "mass_error": rep.mass_error, "relax_ratio": rep.relax_ratio,
            "interface_shift": rep.interface_shift, "interface_limit": rep.interface_limit,
            "seconds": rep.seconds_surrogate, "projected": bool(rep.projected)}


def lbm_project_workspace_bytes(grid) -> int:
    """Device scratch bytes of lbm_project_solenoidal on grid (nx, ny, nz); -1 if invalid."""
    return int(load().lbm_project_workspace_bytes((ctypes.c_int * 3)(*[int(v) for v in grid])))


def lbm_project_solenoidal(u_ptr, grid, work_ptr, work_bytes, stream=None) -> int:
    """The divergence-free part of the periodic velocity at u_ptr (device FP32 [3][nz][ny][nx]),
    in place, with caller-owned scratch (raw device pointers in; returns the lbm status)."""
    gr = (ctypes.c_int * 3)(*[int(v) for v in grid])
    return int(load().lbm_project_solenoidal(ctypes.c_void_p(u_ptr), gr, ctypes.c_void_p(work_ptr), int(work_bytes),
                                             stream))
