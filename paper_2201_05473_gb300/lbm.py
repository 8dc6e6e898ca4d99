"""ctypes binding of the C ABI in ``include/pwfa_lbm.h``.

Argument marshalling only: every step of the method runs in the CUDA kernels
of ``libpwfa_lbm.so``. PyTorch supplies device memory for exported arrays and
the CUDA stream. There is no CPU fallback: loading fails loudly if the library
is missing or cannot be built.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpwfa_lbm.so")

PWFA_OK = 0
ERRORS = {-1: "PWFA_ERR_PARAM", -2: "PWFA_ERR_CUDA", -3: "PWFA_ERR_UNSTABLE",
          -4: "PWFA_ERR_TIMEOUT", -5: "PWFA_ERR_ALLOC", -6: "PWFA_ERR_STATE"}

FIELD_N = 1 << 0
FIELD_UX, FIELD_UY, FIELD_UZ = 1 << 1, 1 << 2, 1 << 3
FIELD_EX, FIELD_EY, FIELD_EZ = 1 << 4, 1 << 5, 1 << 6
FIELD_BX, FIELD_BY, FIELD_BZ = 1 << 7, 1 << 8, 1 << 9
FIELD_JX, FIELD_JY, FIELD_JZ = 1 << 10, 1 << 11, 1 << 12
FIELD_PX, FIELD_PY, FIELD_PZ = 1 << 13, 1 << 14, 1 << 15
RAW_YEE = 1 << 31


class Params(ctypes.Structure):
    """Mirror of ``pwfa_lbm_params``."""
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("tau", ctypes.c_double),
        ("collision", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("boundary", ctypes.c_int32), ("couple", ctypes.c_int32),
        ("n0", ctypes.c_double),
        ("profile", ctypes.POINTER(ctypes.c_double)), ("n_profile", ctypes.c_int32),
        ("profile_rmax", ctypes.c_double),
        ("alpha", ctypes.c_double), ("sigma_r", ctypes.c_double), ("sigma_z", ctypes.c_double),
        ("z0", ctypes.c_double), ("n_floor", ctypes.c_double),
        ("moving_window", ctypes.c_int32), ("window_z", ctypes.c_double),
        ("driver", ctypes.c_int32),
    ]


class AxiParams(ctypes.Structure):
    """Mirror of ``pwfa_axi_params``."""
    _fields_ = [
        ("nz", ctypes.c_int32), ("nr", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("tau", ctypes.c_double),
        ("collision", ctypes.c_int32), ("couple", ctypes.c_int32),
        ("n0", ctypes.c_double),
        ("alpha", ctypes.c_double), ("sigma_r", ctypes.c_double), ("sigma_z", ctypes.c_double),
        ("z0", ctypes.c_double), ("n_floor", ctypes.c_double),
    ]


class LBMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

EXPORTS = ("pwfa_lbm_create", "pwfa_lbm_step", "pwfa_lbm_fields", "pwfa_lbm_get_state",
           "pwfa_lbm_set_state", "pwfa_lbm_steps_done", "pwfa_lbm_set_stream",
           "pwfa_lbm_destroy", "pwfa_lbm_last_error", "pwfa_lbm_profile", "pwfa_lbm_kernel_times",
           "pwfa_lbm_set_launch", "pwfa_lbm_get_launch", "pwfa_lbm_autotune",
           "pwfa_lbm_diag_noalloc", "pwfa_lbm_record", "pwfa_lbm_adjoint_step", "pwfa_lbm_witness_loss", "pwfa_lbm_set_batching",
           "pwfa_lbm_set_field_fusion",
           "pwfa_lbm_step_diag", "pwfa_lbm_linecut", "pwfa_lbm_set_fluid_variant", "pwfa_lbm_get_fluid_variant",
           "pwfa_lbm_window_planes", "pwfa_axi_create", "pwfa_axi_step", "pwfa_axi_fields",
           "pwfa_axi_get_source", "pwfa_axi_set_source", "pwfa_axi_steps_done", "pwfa_axi_profile",
           "pwfa_axi_kernel_times", "pwfa_axi_destroy", "pwfa_lbm_set_particles", "pwfa_lbm_get_particles")


def load(build: bool = True):
    """Load ``libpwfa_lbm.so`` (building it with nvcc first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build:
            from .build import build as _build
            _build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is missing; run paper_2201_05473_gb300.build")
        lib = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        fp, dp = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)
        lib.pwfa_lbm_create.argtypes = [ctypes.POINTER(Params), i32, vp, ctypes.POINTER(vp)]
        lib.pwfa_lbm_step.argtypes = [vp, i32]
        lib.pwfa_lbm_fields.argtypes = [vp, i32, ctypes.c_uint32, vp, i64, dp]
        lib.pwfa_lbm_get_state.argtypes = [vp, i32, vp, vp, vp]
        lib.pwfa_lbm_set_state.argtypes = [vp, i32, vp, vp, vp]
        lib.pwfa_lbm_steps_done.argtypes = [vp, i32]
        lib.pwfa_lbm_steps_done.restype = i64
        lib.pwfa_lbm_window_planes.argtypes = [vp, i32]
        lib.pwfa_lbm_window_planes.restype = i64
        lib.pwfa_axi_create.argtypes = [ctypes.POINTER(AxiParams), vp, ctypes.POINTER(vp)]
        lib.pwfa_axi_step.argtypes = [vp, i32]
        lib.pwfa_axi_fields.argtypes = [vp, vp]
        lib.pwfa_axi_get_source.argtypes = [vp, vp]
        lib.pwfa_axi_set_source.argtypes = [vp, vp]
        lib.pwfa_axi_steps_done.argtypes = [vp]
        lib.pwfa_axi_steps_done.restype = i64
        lib.pwfa_axi_profile.argtypes = [vp, i32]
        lib.pwfa_axi_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
        lib.pwfa_axi_destroy.argtypes = [vp]
        lib.pwfa_lbm_set_particles.argtypes = [vp, i32, i64, vp, ctypes.c_double]
        lib.pwfa_lbm_set_particles.restype = ctypes.c_int
        lib.pwfa_lbm_get_particles.argtypes = [vp, i32, vp]
        lib.pwfa_lbm_get_particles.restype = ctypes.c_int
        for name in ("pwfa_axi_create", "pwfa_axi_step", "pwfa_axi_fields", "pwfa_axi_get_source",
                     "pwfa_axi_set_source", "pwfa_axi_profile", "pwfa_axi_kernel_times", "pwfa_axi_destroy"):
            getattr(lib, name).restype = ctypes.c_int
        lib.pwfa_lbm_set_stream.argtypes = [vp, vp]
        lib.pwfa_lbm_destroy.argtypes = [vp]
        lib.pwfa_lbm_profile.argtypes = [vp, i32]
        lib.pwfa_lbm_kernel_times.argtypes = [vp, dp, ctypes.POINTER(i64)]
        lib.pwfa_lbm_set_launch.argtypes = [vp, i32, i32, i32]
        lib.pwfa_lbm_get_launch.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.pwfa_lbm_autotune.argtypes = [vp, i32]
        lib.pwfa_lbm_set_fluid_variant.argtypes = [vp, i32, i32]
        lib.pwfa_lbm_set_fluid_variant.restype = ctypes.c_int
        lib.pwfa_lbm_get_fluid_variant.argtypes = [vp, i32, ctypes.POINTER(i32)]
        lib.pwfa_lbm_get_fluid_variant.restype = ctypes.c_int
        lib.pwfa_lbm_diag_noalloc.argtypes = [i32, i32, i32, ctypes.c_double, ctypes.c_double,
                                              vp, vp, vp, vp, vp]
        lib.pwfa_lbm_diag_noalloc.restype = ctypes.c_int
        lib.pwfa_lbm_record.argtypes = [vp, i32, i32, i32]
        lib.pwfa_lbm_record.restype = ctypes.c_int
        lib.pwfa_lbm_adjoint_step.argtypes = [vp, i32, vp, i32, i32, dp, i32]
        lib.pwfa_lbm_witness_loss.argtypes = [vp, i32, dp]
        lib.pwfa_lbm_witness_loss.restype = ctypes.c_int
        lib.pwfa_lbm_adjoint_step.restype = ctypes.c_int
        lib.pwfa_lbm_linecut.argtypes = [vp, i32, ctypes.c_double, ctypes.c_double, vp, i64, dp]
        lib.pwfa_lbm_linecut.restype = ctypes.c_int
        lib.pwfa_lbm_step_diag.argtypes = [vp, i32, dp]
        lib.pwfa_lbm_step_diag.restype = ctypes.c_int
        lib.pwfa_lbm_set_batching.argtypes = [vp, i32]
        lib.pwfa_lbm_set_batching.restype = ctypes.c_int
        lib.pwfa_lbm_set_field_fusion.argtypes = [vp, i32]
        lib.pwfa_lbm_set_field_fusion.restype = ctypes.c_int
        lib.pwfa_lbm_last_error.restype = ctypes.c_char_p
        for name in ("pwfa_lbm_create", "pwfa_lbm_step", "pwfa_lbm_fields", "pwfa_lbm_get_state",
                     "pwfa_lbm_set_state", "pwfa_lbm_set_stream", "pwfa_lbm_destroy",
                     "pwfa_lbm_profile", "pwfa_lbm_kernel_times", "pwfa_lbm_set_launch",
                     "pwfa_lbm_get_launch", "pwfa_lbm_autotune"):
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
        return lib


def _check(rc: int):
    if rc != PWFA_OK:
        raise LBMError(rc, _lib.pwfa_lbm_last_error().decode())


def params_of(w: W.Workload):
    """Fill a ``Params`` from a workload; returns (params, keep-alive arrays)."""
    keep = []
    p = Params()
    p.nx, p.ny, p.nz = w.nx, w.ny, w.nz
    p.dx, p.dt, p.tau = w.dx, w.dt, w.tau
    p.collision, p.storage, p.boundary, p.couple = w.collision, w.storage, w.boundary, w.couple
    p.n0 = w.n0
    if w.profile is not None:
        prof = np.ascontiguousarray(w.profile, dtype=np.float64)
        keep.append(prof)
        p.profile = prof.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        p.n_profile = len(prof)
        p.profile_rmax = w.profile_rmax
    p.alpha, p.sigma_r, p.sigma_z, p.z0 = w.alpha, w.sigma_r, w.sigma_z, w.z0
    p.n_floor = w.n_floor
    p.moving_window, p.window_z = int(w.moving_window), w.window_z
    p.driver = int(w.driver)
    return p, keep


def _ptr(t):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        assert t.flags.c_contiguous
        return ctypes.c_void_p(t.ctypes.data)
    assert t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


class Simulation:
    """One or more instances advanced together through the C ABI."""

    def __init__(self, works, stream=None):
        import torch
        self._torch = torch
        self._lib = load()
        if isinstance(works, W.Workload):
            works = [works]
        self.works = list(works)
        arr = (Params * len(self.works))()
        keep = []
        for i, w in enumerate(self.works):
            arr[i], k = params_of(w)
            keep += k
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(self._lib.pwfa_lbm_create(arr, len(self.works), ctypes.c_void_p(stream.cuda_stream),
                                         ctypes.byref(h)))
        self._h = h

    # -- lifecycle
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pwfa_lbm_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- stepping
    def step(self, n: int = 1):
        _check(self._lib.pwfa_lbm_step(self._h, int(n)))

    def step_diag(self, n: int = 1, out=None) -> np.ndarray:
        """Advance n steps; FP64 diagnostics of the state entering the last
        step, fused into it ([n_instances][8], or into a caller-owned host
        float64 buffer)."""
        if out is None:
            out = np.zeros((len(self.works), 8), dtype=np.float64)
        _check(self._lib.pwfa_lbm_step_diag(self._h, int(n),
                                            ctypes.cast(_ptr(out), ctypes.POINTER(ctypes.c_double))))
        return out

    def steps_done(self, instance: int = 0) -> int:
        r = self._lib.pwfa_lbm_steps_done(self._h, instance)
        if r < 0:
            _check(int(r))
        return int(r)

    def set_particles(self, xp, weight: float, instance: int = 0):
        """PIC driver: xp[6][n] = x, y, z at t_{n+1/2}, p_x, p_y, p_z at t_n."""
        t = self._torch
        a = xp.contiguous().to(t.float32) if isinstance(xp, t.Tensor) else \
            t.from_numpy(np.ascontiguousarray(xp, dtype=np.float32))
        self._np = getattr(self, "_np", {})
        self._np[instance] = int(a.shape[1])
        _check(self._lib.pwfa_lbm_set_particles(self._h, instance, int(a.shape[1]), _ptr(a), float(weight)))

    def get_particles(self, instance: int = 0):
        n = getattr(self, "_np", {}).get(instance, 0)
        out = self._torch.empty((6, n), dtype=self._torch.float32, device="cuda")
        _check(self._lib.pwfa_lbm_get_particles(self._h, instance, _ptr(out)))
        return out

    def window_planes(self, instance: int = 0) -> int:
        """Planes the moving window has advanced (box node k sits at lab
        z = (k + W) dx)."""
        r = self._lib.pwfa_lbm_window_planes(self._h, instance)
        if r < 0:
            _check(int(r))
        return int(r)

    def shape(self, instance: int = 0):
        if not 0 <= instance < len(self.works):
            raise LBMError(-1, f"instance {instance} out of range (0..{len(self.works) - 1})")
        w = self.works[instance]
        return (w.nz, w.ny, w.nx)

    # -- exports
    def fields(self, mask: int, instance: int = 0, out=None):
        """Selected fields as a [n_bits][z][y][x] float32 tensor (device unless
        ``out`` is a host tensor/array)."""
        torch = self._torch
        nb = bin(mask & 0xFFFF).count("1")
        shp = (nb,) + self.shape(instance)
        if out is None:
            out = torch.empty(shp, dtype=torch.float32, device="cuda")
        n_el = int(np.prod(shp))
        _check(self._lib.pwfa_lbm_fields(self._h, instance, mask, _ptr(out), n_el, None))
        return out

    def diag(self, instance: int = 0, check: bool = True) -> np.ndarray:
        d = np.zeros(8, dtype=np.float64)
        rc = self._lib.pwfa_lbm_fields(self._h, instance, 0, None, 0,
                                       d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if check or rc != -3:
            _check(rc)
        return d

    def linecut(self, r: float = 0.0, n_star: float = 0.95, instance: int = 0):
        """(n[z], E_z[z], bubble length) along z at offset r from the axis."""
        w = self.works[instance] if 0 <= instance < len(self.works) else None
        if w is None:
            raise LBMError(-1, f"instance {instance} out of range")
        out = np.zeros(2 * w.nz, dtype=np.float32)
        lb = ctypes.c_double()
        _check(self._lib.pwfa_lbm_linecut(self._h, instance, float(r), float(n_star), _ptr(out), out.size,
                                          ctypes.byref(lb)))
        return out[:w.nz], out[w.nz:], lb.value

    def diag_into(self, host_buf, instance: int = 0):
        """FP64 diagnostics into a caller-owned host float64 tensor/array of 8."""
        ptr = _ptr(host_buf)
        rc = self._lib.pwfa_lbm_fields(self._h, instance, 0, None, 0,
                                       ctypes.cast(ptr, ctypes.POINTER(ctypes.c_double)))
        _check(rc)

    def set_launch(self, bx: int, by: int, instance: int = 0):
        _check(self._lib.pwfa_lbm_set_launch(self._h, instance, bx, by))

    def get_launch(self, instance: int = 0):
        bx, by = ctypes.c_int32(), ctypes.c_int32()
        _check(self._lib.pwfa_lbm_get_launch(self._h, instance, ctypes.byref(bx), ctypes.byref(by)))
        return bx.value, by.value

    DIRECT, STAGED = 0, 1

    def set_stream(self, stream):
        """Queue all later work on another torch.cuda.Stream (ordered after
        the work already queued on the current one)."""
        _check(self._lib.pwfa_lbm_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)))
        self.stream = stream

    def set_fluid_variant(self, variant: int, instance: int = 0):
        _check(self._lib.pwfa_lbm_set_fluid_variant(self._h, instance, int(variant)))

    def get_fluid_variant(self, instance: int = 0) -> int:
        v = ctypes.c_int32()
        _check(self._lib.pwfa_lbm_get_fluid_variant(self._h, instance, ctypes.byref(v)))
        return v.value

    def autotune(self, reps: int = 3):
        _check(self._lib.pwfa_lbm_autotune(self._h, reps))

    def record(self, nsteps: int, ckpt_every: int = 0, instance: int = 0):
        """Reset to t = 0 and run nsteps keeping checkpoints for the adjoint."""
        _check(self._lib.pwfa_lbm_record(self._h, instance, int(nsteps), int(ckpt_every)))

    def adjoint_step(self, seed_E=None, nsteps: int = 0, ckpt_every: int = 0, instance: int = 0) -> np.ndarray:
        """Gradient with respect to (alpha, sigma_r, sigma_z, profile...) of
        sum(seed_E * E) (seed_E: [3][z][y][x] float32), or of the built-in
        witness loss when seed_E is None, after the recorded steps; nsteps >= 1
        records that many steps first unless they are already recorded."""
        torch = self._torch
        if seed_E is not None:
            if isinstance(seed_E, np.ndarray):
                seed_E = torch.from_numpy(np.ascontiguousarray(seed_E, dtype=np.float32))
            seed_E = seed_E.contiguous().to(torch.float32)
        w = self.works[instance]
        ng = 3 + (0 if w.profile is None else len(w.profile))
        g = np.zeros(ng, dtype=np.float64)
        _check(self._lib.pwfa_lbm_adjoint_step(self._h, instance, _ptr(seed_E), int(nsteps), int(ckpt_every),
                                               g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ng))
        return g

    def witness_loss(self, instance: int = 0) -> float:
        """The built-in gradient objective -mean(E_z over the witness slab)
        at the current step, reduced in FP64 by the library."""
        v = ctypes.c_double()
        _check(self._lib.pwfa_lbm_witness_loss(self._h, instance, ctypes.byref(v)))
        return v.value

    def profile(self, enable: bool = True):
        _check(self._lib.pwfa_lbm_profile(self._h, 1 if enable else 0))

    KERNELS = ("faraday", "fluid", "ampere", "aux", "adj_fluid", "adj_field")

    def set_batching(self, enable: bool = True):
        _check(self._lib.pwfa_lbm_set_batching(self._h, 1 if enable else 0))

    FUSION_OFF, FUSION_AUTO, FUSION_ON = 0, 1, 2

    def set_field_fusion(self, mode: int = 1):
        """Ampere fused with the next step's Faraday: FUSION_OFF, FUSION_AUTO
        (large grids; the default) or FUSION_ON."""
        _check(self._lib.pwfa_lbm_set_field_fusion(self._h, int(mode)))

    def kernel_times(self):
        """(ms, launches) per kernel kind since the previous call."""
        ms = np.zeros(len(self.KERNELS), dtype=np.float64)
        n = np.zeros(len(self.KERNELS), dtype=np.int64)
        _check(self._lib.pwfa_lbm_kernel_times(
            self._h, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return dict(zip(self.KERNELS, ms)), dict(zip(self.KERNELS, n.tolist()))

    def get_state(self, instance: int = 0, device: bool = True):
        torch = self._torch
        shp = self.shape(instance)
        kw = dict(dtype=torch.float32, device="cuda" if device else "cpu")
        f = torch.empty((4, 19) + shp, **kw)
        E = torch.empty((3,) + shp, **kw)
        B = torch.empty((3,) + shp, **kw)
        _check(self._lib.pwfa_lbm_get_state(self._h, instance, _ptr(f), _ptr(E), _ptr(B)))
        return f, E, B

    def set_state(self, f=None, E=None, B=None, instance: int = 0):
        torch = self._torch
        conv = lambda a: None if a is None else (
            a.contiguous().to(torch.float32) if isinstance(a, torch.Tensor)
            else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)))
        f, E, B = conv(f), conv(E), conv(B)
        _check(self._lib.pwfa_lbm_set_state(self._h, instance, _ptr(f), _ptr(E), _ptr(B)))


class AxiSimulation:
    """The 2D-axisymmetric (z, r) form through the ``pwfa_axi_*`` C ABI.

    Nodes (z_k = k dx, r_j = (j - 1/2) dx); row 0 mirrors the axis, row nr - 1
    and the z planes 0, nz - 1 are boundary nodes. Arrays are [..][z][r]."""

    KERNELS = ("faraday", "moments", "fluid", "ampere")

    def __init__(self, w: "W.AxiWorkload", stream=None):
        import torch
        self._torch = torch
        self._lib = load()
        self.work = w
        p = AxiParams(w.nz, w.nr, w.dx, w.dt, w.tau, w.collision, w.couple, w.n0, w.alpha, w.sigma_r,
                      w.sigma_z, w.z0, w.n_floor)
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(self._lib.pwfa_axi_create(ctypes.byref(p), ctypes.c_void_p(stream.cuda_stream), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.pwfa_axi_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, n: int = 1):
        _check(self._lib.pwfa_axi_step(self._h, int(n)))

    def steps_done(self) -> int:
        r = self._lib.pwfa_axi_steps_done(self._h)
        if r < 0:
            _check(int(r))
        return int(r)

    def fields(self):
        """[6][nz][nr] device tensor: n, beta_z, beta_r, E_z, E_r, B_theta (raw Yee)."""
        out = self._torch.empty((6, self.work.nz, self.work.nr), dtype=self._torch.float32, device="cuda")
        _check(self._lib.pwfa_axi_fields(self._h, _ptr(out)))
        return out

    def get_source(self):
        out = self._torch.empty((3, 9, self.work.nz, self.work.nr), dtype=self._torch.float32, device="cuda")
        _check(self._lib.pwfa_axi_get_source(self._h, _ptr(out)))
        return out

    def set_source(self, fs):
        t = self._torch
        a = fs.contiguous().to(t.float32) if isinstance(fs, t.Tensor) else \
            t.from_numpy(np.ascontiguousarray(fs, dtype=np.float32))
        _check(self._lib.pwfa_axi_set_source(self._h, _ptr(a)))

    def profile(self, enable: bool = True):
        _check(self._lib.pwfa_axi_profile(self._h, 1 if enable else 0))

    def kernel_times(self):
        ms = np.zeros(4, dtype=np.float64)
        n = np.zeros(4, dtype=np.int64)
        _check(self._lib.pwfa_axi_kernel_times(
            self._h, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
            n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return dict(zip(self.KERNELS, ms)), dict(zip(self.KERNELS, n.tolist()))
