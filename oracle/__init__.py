"""FP64 CPU oracle of the difference-free conservative phase-field LBM (arXiv:2407.12263).

TEST INFRASTRUCTURE. Only the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package. The product path (the CUDA
library under ``paper_2407_12263_gb300``) never imports it, and the two share no code.

The arithmetic lives in ``lbm_oracle.c`` (plain C99, FP64, optional OpenMP over z);
this module compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "lbm_oracle.c"
_HDR = _HERE / "lbm_oracle.h"
_BUILD = _HERE / "_build"
_LIB = _BUILD / "liblbm_oracle.so"

CS2 = 1.0 / 3.0

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> Path:
    """Compile the oracle into ``oracle/_build/liblbm_oracle.so`` (gcc, -O2, OpenMP)."""
    _BUILD.mkdir(exist_ok=True)
    newest = max(_SRC.stat().st_mtime, _HDR.stat().st_mtime)
    if not force and _LIB.exists() and _LIB.stat().st_mtime >= newest:
        return _LIB
    tmp = _BUILD / f"liblbm_oracle.{os.getpid()}.so"
    base = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-o", str(tmp), str(_SRC), "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(str(build()))
    lib.oracle_lattice.argtypes = [ctypes.c_int, _ip, _ip, _dp]
    lib.oracle_lax_wendroff.argtypes = [ctypes.c_double] * 4
    lib.oracle_lax_wendroff.restype = ctypes.c_double
    lib.oracle_css_tensor.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp]
    lib.oracle_feq.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _dp, _dp, ctypes.c_int, _dp]
    lib.oracle_geq.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_double, _dp]
    lib.oracle_forcing.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp, _dp]
    lib.oracle_isotropic_gradient.argtypes = [ctypes.c_int] * 4 + [_dp, _dp]
    lib.oracle_create.argtypes = ([ctypes.c_int] * 4 + [ctypes.c_double] * 7 + [_dp, ctypes.c_double]
                                  + [ctypes.c_int] * 4)
    lib.oracle_create.restype = ctypes.c_void_p
    lib.oracle_destroy.argtypes = [ctypes.c_void_p]
    lib.oracle_set_walls.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.oracle_tau_phi.argtypes = [ctypes.c_void_p]
    lib.oracle_tau_phi.restype = ctypes.c_double
    lib.oracle_macroscopic_cell.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
    lib.oracle_collide_cell.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp, _dp]
    lib.oracle_init_phi.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_double]
    lib.oracle_init_fields.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, ctypes.c_double]
    lib.oracle_step.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.oracle_moments.argtypes = [ctypes.c_void_p] + [_dp] * 5
    lib.oracle_mass.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.oracle_get_pops.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.oracle_set_pops.argtypes = [ctypes.c_void_p, _dp, _dp]
    lib.oracle_set_num_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_num_threads.restype = None
    _lib = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _vec(v, n=3):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(n))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the following oracle calls (results do not depend on it)."""
    _load().oracle_set_num_threads(int(n))


# --------------------------------------------------------------------------
# Building blocks (each is the function the full scheme calls).
# --------------------------------------------------------------------------
def lattice(Q: int):
    """(d, e[Q,3], t[Q]) of D2Q9 (Sec. 2.2) or D3Q19."""
    d = ctypes.c_int()
    e = np.zeros(3 * Q, dtype=np.int32)
    t = np.zeros(Q)
    if _load().oracle_lattice(Q, ctypes.byref(d), e.ctypes.data_as(_ip), _ptr(t)):
        raise ValueError(f"unknown lattice Q={Q}")
    return d.value, e.reshape(Q, 3).astype(np.int64), t


def lax_wendroff(c, at_minus, at_x, at_plus) -> float:
    return float(_load().oracle_lax_wendroff(c, at_minus, at_x, at_plus))


def css_tensor(d, sigma, grad_norm, n):
    out = np.zeros(9)
    _load().oracle_css_tensor(d, sigma, grad_norm, _ptr(_vec(n)), _ptr(out))
    return out.reshape(3, 3)


def feq(Q, p, rho, u, pis, pis_sign=-1):
    out = np.zeros(Q)
    _load().oracle_feq(Q, p, rho, _ptr(_vec(u)), _ptr(_vec(pis, 9)), pis_sign, _ptr(out))
    return out


def geq(Q, phi, u, S, src_scale):
    out = np.zeros(Q)
    _load().oracle_geq(Q, phi, _ptr(_vec(u)), _ptr(_vec(S)), src_scale, _ptr(out))
    return out


def forcing(Q, rho, u, grad_rho, G):
    Si = np.zeros(Q)
    Ri = np.zeros(Q)
    _load().oracle_forcing(Q, rho, _ptr(_vec(u)), _ptr(_vec(grad_rho)), _ptr(_vec(G)), _ptr(Si), _ptr(Ri))
    return Si, Ri


def isotropic_gradient(Q, field):
    """Isotropic central-difference gradient of a periodic field shaped (nz, ny, nx)."""
    field = np.ascontiguousarray(field, dtype=np.float64)
    nz, ny, nx = field.shape
    grad = np.zeros((3,) + field.shape)
    _load().oracle_isotropic_gradient(Q, nx, ny, nz, _ptr(field), _ptr(grad))
    return grad


MACRO_FIELDS = {"phi": 0, "rho": 1, "u": slice(2, 5), "K1": slice(5, 8), "n": slice(8, 11),
                "S": slice(11, 14), "grad_phi": slice(14, 17), "grad_rho": slice(17, 20), "p": 20}


class Oracle:
    """The scheme on a periodic grid; arrays are shaped (nz, ny, nx) (planes first for vectors)."""

    def __init__(self, Q, grid, tau_f, tau_g, M, xi, sigma, rho_ratio=1.0, mu_ratio=1.0,
                 body_force=(0.0, 0.0, 0.0), courant=0.997, scheme=0, pis_sign=-1,
                 half_force_sign=1, geq_source_tau=1, walls=0):
        nx, ny, nz = grid
        self.Q, self.grid = Q, (nx, ny, nz)
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        lib = _load()
        self._h = lib.oracle_create(Q, nx, ny, nz, tau_f, tau_g, M, xi, sigma, rho_ratio, mu_ratio,
                                    _ptr(_vec(body_force)), courant, scheme, pis_sign,
                                    half_force_sign, geq_source_tau)
        if not self._h:
            raise ValueError("oracle_create rejected the arguments")
        if lib.oracle_set_walls(self._h, int(walls)) != 0:
            raise ValueError(f"invalid wall mask {walls}")
        self.tau_phi = float(lib.oracle_tau_phi(self._h))
        self.walls = int(walls)

    def close(self):
        if getattr(self, "_h", None):
            _load().oracle_destroy(self._h)
            self._h = None

    __del__ = close

    def init_phi(self, phi0, u0=None, p0=CS2, p=None):
        """Initial state; p (a pressure field, optional) replaces the uniform p0 in f^eq."""
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(self.shape)
        u0 = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64).reshape((3,) + self.shape)
        p = None if p is None else np.ascontiguousarray(p, dtype=np.float64).reshape(self.shape)
        _load().oracle_init_fields(self._h, _ptr(phi0), _ptr(u0), _ptr(p), p0)

    def step(self, n=1):
        if _load().oracle_step(self._h, int(n)) != 0:
            raise RuntimeError("oracle_step before init")

    def moments(self):
        phi = np.zeros(self.shape)
        p = np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        _load().oracle_moments(self._h, _ptr(phi), _ptr(p), _ptr(u), None, None)
        return phi, p, u

    def gradients(self):
        gphi = np.zeros((3,) + self.shape)
        n = np.zeros((3,) + self.shape)
        _load().oracle_moments(self._h, None, None, None, _ptr(gphi), _ptr(n))
        return gphi, n

    def mass(self):
        a, b = ctypes.c_double(), ctypes.c_double()
        _load().oracle_mass(self._h, ctypes.byref(a), ctypes.byref(b))
        return a.value, b.value

    def get_pops(self):
        f = np.zeros((self.Q,) + self.shape)
        g = np.zeros((self.Q,) + self.shape)
        _load().oracle_get_pops(self._h, _ptr(f), _ptr(g))
        return f, g

    def set_pops(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape((self.Q,) + self.shape)
        g = np.ascontiguousarray(g, dtype=np.float64).reshape((self.Q,) + self.shape)
        _load().oracle_set_pops(self._h, _ptr(f), _ptr(g))

    def restart_from_coarse(self, coarse, factor, p0=CS2):
        """Replace the state by the restart from coarse fields (the surrogate's hand-over to the
        lattice; no counterpart in the paper). See ``oracle.restart``: trilinear upsampling of
        (phi, u, v, w, p), phi clamped to [-1, 1.5], the initial-state construction of reading R9
        (``init_phi`` with the pressure field), then sum phi set back to its value before."""
        from . import restart as _restart

        _restart.restart_from_coarse(self, coarse, factor, p0)

    def macroscopic_cell(self, fbar, g, fd_grad=None):
        out = np.zeros(21)
        _load().oracle_macroscopic_cell(self._h, _ptr(_vec(fbar, self.Q)), _ptr(_vec(g, self.Q)),
                                        None if fd_grad is None else _ptr(_vec(fd_grad)), _ptr(out))
        return {k: (out[v].copy() if isinstance(v, slice) else float(out[v])) for k, v in MACRO_FIELDS.items()}

    def collide_cell(self, fbar, g, macro: dict):
        packed = np.zeros(21)
        for k, v in MACRO_FIELDS.items():
            packed[v] = macro[k]
        fs = np.zeros(self.Q)
        gs = np.zeros(self.Q)
        _load().oracle_collide_cell(self._h, _ptr(_vec(fbar, self.Q)), _ptr(_vec(g, self.Q)),
                                    _ptr(packed), _ptr(fs), _ptr(gs))
        return fs, gs
