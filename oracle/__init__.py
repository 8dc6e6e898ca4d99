"""FP64 CPU oracle of the lattice-Boltzmann plasma-wakefield step.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference arm of ``bench.py`` may import this package. The GPU
library never calls it and shares no code with it.

The arithmetic lives in ``pwfa_oracle.cpp`` (plain loops in double precision,
one function per step of the method: Faraday, collision + source, streaming,
Eq. 14 boundary, Ampere). This module only builds that file with g++ and
marshals NumPy arrays through ctypes.

Array layouts of every accessor: populations ``[lattice][q][z][y][x]``, Yee
fields ``[component][z][y][x]`` (E_x at (i+1/2, j, k), B_x at (i, j+1/2, k+1/2)
and cyclic), node quantities ``[component][z][y][x]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pwfa_oracle.cpp")
_SRCS = [_SRC, os.path.join(_HERE, "axi_oracle.cpp")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

COLL_BGK, COLL_REG, COLL_NONE = 0, 1, 2
BND_OPEN, BND_PERIODIC = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (g++, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(s) for s in _SRCS)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-Wall",
           "-o", tmp] + _SRCS
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("tau", ctypes.c_double),
        ("collision", ctypes.c_int32), ("boundary", ctypes.c_int32), ("couple", ctypes.c_int32),
        ("n0", ctypes.c_double),
        ("profile", ctypes.POINTER(ctypes.c_double)), ("n_profile", ctypes.c_int32),
        ("profile_rmax", ctypes.c_double),
        ("alpha", ctypes.c_double), ("sigma_r", ctypes.c_double), ("sigma_z", ctypes.c_double),
        ("z0", ctypes.c_double),
        ("n_floor", ctypes.c_double),
        ("moving_window", ctypes.c_int32), ("window_z", ctypes.c_double),
        ("driver", ctypes.c_int32),
    ]


class _AxiParams(ctypes.Structure):
    _fields_ = [
        ("nz", ctypes.c_int32), ("nr", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("tau", ctypes.c_double),
        ("collision", ctypes.c_int32), ("couple", ctypes.c_int32),
        ("n0", ctypes.c_double),
        ("alpha", ctypes.c_double), ("sigma_r", ctypes.c_double), ("sigma_z", ctypes.c_double),
        ("z0", ctypes.c_double),
        ("n_floor", ctypes.c_double),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.oracle_create.restype = ctypes.c_void_p
            lib.oracle_create.argtypes = [ctypes.POINTER(_Params)]
            lib.oracle_destroy.argtypes = [ctypes.c_void_p]
            lib.oracle_step.argtypes = [ctypes.c_void_p, ctypes.c_int32]
            lib.oracle_step.restype = ctypes.c_int
            lib.oracle_window_planes.restype = ctypes.c_int64
            lib.oracle_window_planes.argtypes = [ctypes.c_void_p]
            lib.oracle_set_source.argtypes = [ctypes.c_void_p, dp]
            lib.oracle_set_particles.argtypes = [ctypes.c_void_p, ctypes.c_int64, dp, ctypes.c_double]
            lib.oracle_get_particles.argtypes = [ctypes.c_void_p, dp]
            lib.oracle_driver_current.argtypes = [ctypes.c_void_p, dp]
            lib.oracle_steps_done.restype = ctypes.c_int64
            lib.oracle_steps_done.argtypes = [ctypes.c_void_p]
            for name in ("oracle_get_f", "oracle_set_f", "oracle_set_equilibrium",
                         "oracle_moments", "oracle_diag"):
                getattr(lib, name).argtypes = [ctypes.c_void_p, dp]
            lib.oracle_get_fields.argtypes = [ctypes.c_void_p, dp, dp]
            lib.oracle_set_fields.argtypes = [ctypes.c_void_p, dp, dp]
            lib.oracle_last_step.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
            lib.oracle_tangent_run.argtypes = [ctypes.POINTER(_Params), ctypes.c_int32, ctypes.c_int32,
                                               dp, dp, dp]
            lib.oracle_tangent_run.restype = ctypes.c_int
            lib.axi_create.restype = ctypes.c_void_p
            lib.axi_create.argtypes = [ctypes.POINTER(_AxiParams)]
            lib.axi_destroy.argtypes = [ctypes.c_void_p]
            lib.axi_step.argtypes = [ctypes.c_void_p, ctypes.c_int32]
            lib.axi_steps_done.restype = ctypes.c_int64
            lib.axi_steps_done.argtypes = [ctypes.c_void_p]
            for name in ("axi_get_f", "axi_set_f", "axi_set_equilibrium", "axi_moments", "axi_get_source",
                         "axi_set_source"):
                getattr(lib, name).argtypes = [ctypes.c_void_p, dp]
            lib.axi_get_fields.argtypes = [ctypes.c_void_p, dp, dp, dp]
            lib.axi_set_fields.argtypes = [ctypes.c_void_p, dp, dp, dp]
            lib.axi_last_current.argtypes = [ctypes.c_void_p, dp, dp]
            lib.oracle_qtilde.restype = ctypes.c_double
            lib.oracle_qtilde.argtypes = [ctypes.c_double] * 5 + [dp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """One FP64 simulation instance (see ``pwfa_oracle.cpp`` for the step)."""

    def __init__(self, nx, ny, nz, dx, dt, tau, collision=COLL_BGK, boundary=BND_OPEN,
                 couple=1, n0=1.0, profile=None, profile_rmax=0.0, alpha=0.0,
                 sigma_r=0.5, sigma_z=0.5, z0=0.0, n_floor=1e-6, moving_window=0, window_z=0.0, driver=0):
        self._lib = _load()
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        prof = None if profile is None else np.ascontiguousarray(profile, dtype=np.float64)
        self._prof = prof
        p = _Params(nx, ny, nz, dx, dt, tau, collision, boundary, couple, n0,
                    _ptr(prof) if prof is not None else None,
                    0 if prof is None else len(prof), profile_rmax,
                    alpha, sigma_r, sigma_z, z0, n_floor, int(moving_window), window_z, int(driver))
        self._h = self._lib.oracle_create(ctypes.byref(p))
        self._np = 0
        if not self._h:
            raise ValueError("oracle_create rejected the parameters")
        self.params = dict(nx=nx, ny=ny, nz=nz, dx=dx, dt=dt, tau=tau, collision=collision,
                           boundary=boundary, couple=couple, n0=n0, alpha=alpha,
                           sigma_r=sigma_r, sigma_z=sigma_z, z0=z0, n_floor=n_floor,
                           moving_window=moving_window, window_z=window_z)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.oracle_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        if self._lib.oracle_step(self._h, int(n)) != 0:
            raise RuntimeError("oracle step failed: a window move needs the streaming source "
                               "(not available after set_f / set_equilibrium)")

    @property
    def window_planes(self) -> int:
        """Planes the moving window has advanced (0 without a window)."""
        return int(self._lib.oracle_window_planes(self._h))

    def set_particles(self, xp: np.ndarray, weight: float):
        """PIC driver: xp[6][n] = x, y, z at t_{n+1/2}, p_x, p_y, p_z at t_n."""
        xp = np.ascontiguousarray(xp, dtype=np.float64)
        self._np = xp.shape[1]
        self._lib.oracle_set_particles(self._h, self._np, _ptr(xp), float(weight))

    def get_particles(self) -> np.ndarray:
        out = np.empty((6, self._np))
        self._lib.oracle_get_particles(self._h, _ptr(out))
        return out

    def driver_current(self) -> np.ndarray:
        out = np.empty((3,) + self.shape)
        self._lib.oracle_driver_current(self._h, _ptr(out))
        return out

    def set_source(self, fs: np.ndarray):
        """Set the streaming source (post-collision populations) and pull the
        pre-collision state from it."""
        fs = np.ascontiguousarray(fs, dtype=np.float64).reshape((4, 19) + self.shape)
        self._lib.oracle_set_source(self._h, _ptr(fs))

    @property
    def steps_done(self) -> int:
        return int(self._lib.oracle_steps_done(self._h))

    def get_f(self) -> np.ndarray:
        out = np.empty((4, 19) + self.shape, dtype=np.float64)
        self._lib.oracle_get_f(self._h, _ptr(out))
        return out

    def set_f(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape((4, 19) + self.shape)
        self._lib.oracle_set_f(self._h, _ptr(f))

    def set_equilibrium(self, A: np.ndarray):
        A = np.ascontiguousarray(A, dtype=np.float64).reshape((4,) + self.shape)
        self._lib.oracle_set_equilibrium(self._h, _ptr(A))

    def get_fields(self):
        E = np.empty((3,) + self.shape, dtype=np.float64)
        B = np.empty((3,) + self.shape, dtype=np.float64)
        self._lib.oracle_get_fields(self._h, _ptr(E), _ptr(B))
        return E, B

    def set_fields(self, E: np.ndarray, B: np.ndarray):
        E = np.ascontiguousarray(E, dtype=np.float64).reshape((3,) + self.shape)
        B = np.ascontiguousarray(B, dtype=np.float64).reshape((3,) + self.shape)
        self._lib.oracle_set_fields(self._h, _ptr(E), _ptr(B))

    def moments(self) -> dict:
        out = np.empty((8,) + self.shape, dtype=np.float64)
        self._lib.oracle_moments(self._h, _ptr(out))
        return {"n": out[0], "beta": out[1:4], "A": out[4:7], "beta_abs": out[7]}

    def last_step(self) -> dict:
        J = np.empty((3,) + self.shape)
        F = np.empty((4,) + self.shape)
        En = np.empty((3,) + self.shape)
        Bn = np.empty((3,) + self.shape)
        self._lib.oracle_last_step(self._h, _ptr(J), _ptr(F), _ptr(En), _ptr(Bn))
        return {"J": J, "F": F, "E_node": En, "B_node": Bn}

    def diag(self) -> np.ndarray:
        out = np.empty(8, dtype=np.float64)
        self._lib.oracle_diag(self._h, _ptr(out))
        return out


class AxiOracle:
    """2D-axisymmetric (z, r) FP64 simulation (see ``axi_oracle.cpp``).

    Nodes (z_k, r_j), z_k = k dx, r_j = (j - 1/2) dx; row 0 mirrors the axis,
    row nr - 1 is the outer boundary row. Arrays are ``[..][z][r]``."""

    def __init__(self, nz, nr, dx, dt, tau, collision=COLL_BGK, couple=1, n0=1.0, alpha=0.0,
                 sigma_r=0.5, sigma_z=0.5, z0=0.0, n_floor=1e-6):
        self._lib = _load()
        self.shape = (nz, nr)
        self.N = nz * nr
        p = _AxiParams(nz, nr, dx, dt, tau, collision, couple, n0, alpha, sigma_r, sigma_z, z0, n_floor)
        self._h = self._lib.axi_create(ctypes.byref(p))
        if not self._h:
            raise ValueError("axi_create rejected the parameters")
        self.params = dict(nz=nz, nr=nr, dx=dx, dt=dt, tau=tau, collision=collision, couple=couple, n0=n0,
                           alpha=alpha, sigma_r=sigma_r, sigma_z=sigma_z, z0=z0, n_floor=n_floor)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.axi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        self._lib.axi_step(self._h, int(n))

    @property
    def steps_done(self) -> int:
        return int(self._lib.axi_steps_done(self._h))

    def radii(self) -> np.ndarray:
        return (np.arange(self.shape[1]) - 0.5) * self.params["dx"]

    def get_f(self) -> np.ndarray:
        out = np.empty((3, 9) + self.shape)
        self._lib.axi_get_f(self._h, _ptr(out))
        return out

    def set_f(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape((3, 9) + self.shape)
        self._lib.axi_set_f(self._h, _ptr(f))

    def set_equilibrium(self, A):
        A = np.ascontiguousarray(A, dtype=np.float64).reshape((3,) + self.shape)
        self._lib.axi_set_equilibrium(self._h, _ptr(A))

    def get_source(self) -> np.ndarray:
        out = np.empty((3, 9) + self.shape)
        self._lib.axi_get_source(self._h, _ptr(out))
        return out

    def set_source(self, fs):
        fs = np.ascontiguousarray(fs, dtype=np.float64).reshape((3, 9) + self.shape)
        self._lib.axi_set_source(self._h, _ptr(fs))

    def get_fields(self):
        Ez, Er, Bt = (np.empty(self.shape) for _ in range(3))
        self._lib.axi_get_fields(self._h, _ptr(Ez), _ptr(Er), _ptr(Bt))
        return Ez, Er, Bt

    def set_fields(self, Ez, Er, Bt):
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape) for a in (Ez, Er, Bt)]
        self._lib.axi_set_fields(self._h, *(_ptr(a) for a in arrs))

    def moments(self) -> dict:
        out = np.empty((6,) + self.shape)
        self._lib.axi_moments(self._h, _ptr(out))
        return {"n": out[0], "beta_z": out[1], "beta_r": out[2], "A": out[3:5], "beta_abs": out[5]}

    def last_current(self):
        Jz, Jr = np.empty(self.shape), np.empty(self.shape)
        self._lib.axi_last_current(self._h, _ptr(Jz), _ptr(Jr))
        return Jz, Jr


def tangent_run(nsteps, dirs, nx, ny, nz, dx, dt, tau, collision=COLL_BGK, boundary=BND_OPEN,
                couple=1, n0=1.0, profile=None, profile_rmax=0.0, alpha=0.0, sigma_r=0.5,
                sigma_z=0.5, z0=0.0, n_floor=1e-6):
    """Raw Yee E after nsteps and its derivatives along dirs ([ndir][3 + n_profile],
    parameters ordered alpha, sigma_r, sigma_z, profile...), by forward-mode
    dual numbers. Returns (E [3][z][y][x], dE [ndir][3][z][y][x])."""
    lib = _load()
    dirs = np.ascontiguousarray(np.atleast_2d(dirs), dtype=np.float64)
    prof = None if profile is None else np.ascontiguousarray(profile, dtype=np.float64)
    p = _Params(nx, ny, nz, dx, dt, tau, collision, boundary, couple, n0,
                _ptr(prof) if prof is not None else None, 0 if prof is None else len(prof),
                profile_rmax, alpha, sigma_r, sigma_z, z0, n_floor, 0, 0.0, 0)
    nd = dirs.shape[0]
    assert dirs.shape[1] == 3 + (0 if prof is None else len(prof))
    E = np.empty((3, nz, ny, nx))
    dE = np.empty((nd, 3, nz, ny, nx))
    if lib.oracle_tangent_run(ctypes.byref(p), int(nsteps), nd, _ptr(dirs), _ptr(E), _ptr(dE)) != 0:
        raise ValueError("oracle_tangent_run failed")
    return E, dE


def qtilde(charge_coulomb, sx, sy, sz, n0_m3):
    """Normalised charge (Eq. 15, read with k_p^3) and alpha = n_b/n0."""
    a = np.zeros(1)
    q = _load().oracle_qtilde(charge_coulomb, sx, sy, sz, n0_m3, _ptr(a))
    return q, float(a[0])
