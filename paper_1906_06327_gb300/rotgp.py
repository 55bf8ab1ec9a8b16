"""ctypes binding of ``librotgp.so`` (the C ABI of ``include/rotgp.h``).

Argument marshalling only: every numerical step runs in the CUDA library.
The library is loaded on first use and a missing or unloadable library is an
error (there is no fallback).  Device memory and streams may come from
PyTorch: pass ``torch.cuda.current_stream().cuda_stream`` as the stream and
CUDA tensors as device buffers.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

ROTGP_OK = 0
ROTGP_EINVAL = -1
ROTGP_ENOMEM = -2
ROTGP_ECUDA = -3
ROTGP_ENONFINITE = -4
ROTGP_EUNSUPPORTED = -5
ROTGP_ETIMEOUT = -6
ROTGP_FP64 = 0
ROTGP_FP32 = 1
ROTGP_SOLVER_THOMAS = 0
ROTGP_SOLVER_STENCIL = 1
ROTGP_SOLVER_FUSED = 2
ROTGP_SOLVER_HYBRID = 3

ERROR_NAMES = {ROTGP_EINVAL: "EINVAL", ROTGP_ENOMEM: "ENOMEM", ROTGP_ECUDA: "ECUDA",
               ROTGP_ENONFINITE: "ENONFINITE", ROTGP_EUNSUPPORTED: "EUNSUPPORTED",
               ROTGP_ETIMEOUT: "ETIMEOUT"}

# Every entry point declared in include/rotgp.h.
EXPORTS = ("rotgp_create", "rotgp_destroy", "rotgp_last_error", "rotgp_set_phys",
           "rotgp_set_omega", "rotgp_init_analytic", "rotgp_init_analytic_field",
           "rotgp_set_psi", "rotgp_get_psi", "rotgp_column_density",
           "rotgp_step_imag", "rotgp_step_real", "rotgp_step_schedule", "rotgp_observables",
           "rotgp_sync",
           "rotgp_info", "rotgp_tune", "rotgp_set_solver", "rotgp_autotune",
           "rotgp_check_bounded_wait",
           "rotgp_profile_enable",
           "rotgp_profile_read",
           "rotgp_observables_noalloc",
           "rotgp_batch_create", "rotgp_batch_destroy", "rotgp_batch_last_error",
           "rotgp_batch_count", "rotgp_batch_context", "rotgp_batch_autotune",
           "rotgp_batch_step", "rotgp_batch_sync", "rotgp_batch_observables",
           "rotgp_batch_converge",
           "rotgp_ws_param_count", "rotgp_ws_create", "rotgp_ws_destroy", "rotgp_ws_last_error",
           "rotgp_ws_set_params", "rotgp_ws_get_params", "rotgp_ws_propose",
           "rotgp_ws_train_step", "rotgp_ws_gradients")


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("h", ctypes.c_double * 3)]


class Phys(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("gamma", "nu", "lam", "g", "omega", "dt")]


class Obs(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("norm", "mu", "energy", "mu_c", "energy_c",
                                                "rms_x", "rms_y", "rms_z", "rms_r",
                                                "max_density", "mu4", "energy4")] + \
               [("step", ctypes.c_longlong), ("vortices", ctypes.c_int), ("flags", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class KStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_longlong),
                ("total_ms", ctypes.c_double), ("bytes_per_launch", ctypes.c_double)]


class SolverInfo(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("halo", ctypes.c_int), ("table_len", ctypes.c_int),
                ("chunk", ctypes.c_int * 3), ("segments", ctypes.c_int * 3),
                ("lines_per_lane", ctypes.c_int * 3), ("ring", ctypes.c_int * 3),
                ("stencil_taps", ctypes.c_int * 3),
                ("warps_per_block", ctypes.c_int * 3), ("fused_xy", ctypes.c_int),
                ("hybrid_cluster", ctypes.c_int * 3),
                ("decay", ctypes.c_double), ("device_bytes", ctypes.c_size_t)]


class RotgpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rotgp error {ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load librotgp.so (building it with nvcc if absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise RuntimeError(f"CUDA library missing: {path}")
            _build.build()
        lib = ctypes.CDLL(path)
        vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)
        lib.rotgp_create.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Phys), ip, vp,
                                     ctypes.POINTER(vp)]
        lib.rotgp_destroy.argtypes = [vp]
        lib.rotgp_destroy.restype = None
        lib.rotgp_last_error.argtypes = [vp]
        lib.rotgp_last_error.restype = ctypes.c_char_p
        lib.rotgp_set_phys.argtypes = [vp, ctypes.POINTER(Phys)]
        lib.rotgp_set_omega.argtypes = [vp, ctypes.c_double]
        lib.rotgp_init_analytic.argtypes = [vp, ip, ip, ctypes.c_ulonglong, ctypes.c_double,
                                            ctypes.c_double]
        lib.rotgp_init_analytic_field.argtypes = [vp, ip, dp, ctypes.c_double, ctypes.c_double]
        lib.rotgp_set_psi.argtypes = [vp, vp, ip, ip, ip]
        lib.rotgp_get_psi.argtypes = [vp, vp, ip, ip]
        lib.rotgp_column_density.argtypes = [vp, dp, ip]
        lib.rotgp_step_imag.argtypes = [vp, ctypes.c_longlong]
        lib.rotgp_step_real.argtypes = [vp, ctypes.c_longlong]
        lib.rotgp_step_schedule.argtypes = [vp, ctypes.c_longlong, ip, dp]
        lib.rotgp_observables.argtypes = [vp, ctypes.POINTER(Obs)]
        lib.rotgp_sync.argtypes = [vp]
        lib.rotgp_info.argtypes = [vp, ctypes.POINTER(SolverInfo)]
        lib.rotgp_tune.argtypes = [vp, ip, ip, ip, ip, ip, ip]
        lib.rotgp_set_solver.argtypes = [vp, ip, ip]
        lib.rotgp_autotune.argtypes = [vp, ip, ctypes.POINTER(ip)]
        lib.rotgp_check_bounded_wait.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
        lib.rotgp_profile_enable.argtypes = [vp, ip]
        lib.rotgp_profile_read.argtypes = [vp, ctypes.POINTER(KStat), ip, ctypes.POINTER(ip)]
        lib.rotgp_observables_noalloc.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Phys), ip,
                                                  vp, vp, ctypes.POINTER(Obs)]
        ll = ctypes.c_longlong
        lib.rotgp_batch_create.argtypes = [ip, ctypes.POINTER(Grid), ctypes.POINTER(Phys), ip, vp,
                                           ctypes.POINTER(vp)]
        lib.rotgp_batch_destroy.argtypes = [vp]
        lib.rotgp_batch_destroy.restype = None
        lib.rotgp_batch_last_error.argtypes = [vp]
        lib.rotgp_batch_last_error.restype = ctypes.c_char_p
        lib.rotgp_batch_count.argtypes = [vp]
        lib.rotgp_batch_context.argtypes = [vp, ip, ctypes.POINTER(vp)]
        lib.rotgp_batch_autotune.argtypes = [vp, ip]
        lib.rotgp_batch_step.argtypes = [vp, ll, ip, ip]
        lib.rotgp_batch_sync.argtypes = [vp]
        lib.rotgp_batch_observables.argtypes = [vp, ctypes.POINTER(Obs)]
        lib.rotgp_batch_converge.argtypes = [vp, ctypes.c_double, ll, ll, ip,
                                             ctypes.POINTER(ll), ctypes.POINTER(ip)]
        lib.rotgp_ws_param_count.argtypes = []
        lib.rotgp_ws_param_count.restype = ll
        lib.rotgp_ws_create.argtypes = [ip, ip, vp, ctypes.POINTER(vp)]
        lib.rotgp_ws_destroy.argtypes = [vp]
        lib.rotgp_ws_destroy.restype = None
        lib.rotgp_ws_last_error.argtypes = [vp]
        lib.rotgp_ws_last_error.restype = ctypes.c_char_p
        fp = ctypes.POINTER(ctypes.c_float)
        lib.rotgp_ws_set_params.argtypes = [vp, fp]
        lib.rotgp_ws_get_params.argtypes = [vp, fp]
        lib.rotgp_ws_propose.argtypes = [vp, ip, dp, ctypes.c_double, ip, ctypes.c_ulonglong, vp,
                                         ip]
        lib.rotgp_ws_train_step.argtypes = [vp, ip, dp, ctypes.c_double, vp, ip, ctypes.c_float,
                                            dp]
        lib.rotgp_ws_gradients.argtypes = [vp, ip, vp, fp, dp, fp]
        _lib = lib
        return lib


def _shape(n) -> tuple:
    return tuple(int(v) + 1 for v in reversed(n))


class Solver:
    """One condensate: ``rotgp_create`` ... ``rotgp_destroy``.

    n: intervals per axis (2 or 3 values), h: spacings, precision "fp32" or
    "fp64", stream: a cudaStream_t as int (0 = default stream).
    """

    def __init__(self, n, h, *, gamma=1.0, nu=1.0, lam=1.0, g=0.0, omega=0.0, dt=1e-3,
                 precision="fp32", stream=0, _borrowed=None):
        self._lib = load()
        self.n, self.h = tuple(int(v) for v in n), tuple(float(v) for v in h)
        self.dim = len(self.n)
        self.fp64 = precision == "fp64"
        grid = Grid(self.dim, (ctypes.c_int * 3)(*(list(self.n) + [0] * (3 - self.dim))),
                    (ctypes.c_double * 3)(*(list(self.h) + [0.0] * (3 - self.dim))))
        self.phys = Phys(gamma, nu, lam, g, omega, dt)
        self._owned = _borrowed is None
        if _borrowed is not None:
            # a context owned by a Batch
            self._h = _borrowed
            return
        handle = ctypes.c_void_p()
        rc = self._lib.rotgp_create(ctypes.byref(grid), ctypes.byref(self.phys),
                                    ROTGP_FP64 if self.fp64 else ROTGP_FP32,
                                    ctypes.c_void_p(int(stream)), ctypes.byref(handle))
        if rc != ROTGP_OK:
            raise RotgpError(rc, self._lib.rotgp_last_error(None).decode())
        self._h = handle

    # -- plumbing
    def _check(self, rc: int):
        if rc != ROTGP_OK:
            raise RotgpError(rc, self._lib.rotgp_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                self._lib.rotgp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def shape(self) -> tuple:
        """Shape of an ABI wave function: (N_z+1,) (N_y+1, N_x+1)."""
        return _shape(self.n)

    @property
    def handle(self) -> int:
        return self._h.value

    # -- physics
    def set_phys(self, **kw):
        p = Phys(*[kw.get(k, getattr(self.phys, k)) for k, _ in Phys._fields_])
        self._check(self._lib.rotgp_set_phys(self._h, ctypes.byref(p)))
        self.phys = p

    def set_omega(self, omega: float):
        self._check(self._lib.rotgp_set_omega(self._h, float(omega)))
        self.phys.omega = float(omega)

    # -- state
    def init_analytic(self, function: int = 1, phase_R=None, d_xy: float = 1.0, d_z: float = 1.0,
                      *, seed=None):
        """Eq. fun.  ``seed``: the library draws R from SplitMix64(seed)
        (``rotgp_init_analytic``); else ``phase_R`` is the (N_y+1, N_x+1)
        array R or None (``rotgp_init_analytic_field``)."""
        if seed is not None:
            if phase_R is not None:
                raise ValueError("give either seed or phase_R")
            self._check(self._lib.rotgp_init_analytic(self._h, int(function), 1,
                                                      int(seed) & 0xFFFFFFFFFFFFFFFF,
                                                      float(d_xy), float(d_z)))
            return
        ptr = None
        if phase_R is not None:
            phase_R = np.ascontiguousarray(phase_R, dtype=np.float64)
            if phase_R.shape != (self.n[1] + 1, self.n[0] + 1):
                raise ValueError("phase_R must have shape (N_y+1, N_x+1)")
            ptr = phase_R.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        self._check(self._lib.rotgp_init_analytic_field(self._h, int(function), ptr,
                                                        float(d_xy), float(d_z)))

    def set_psi(self, psi, normalise: bool = False):
        """psi: numpy complex64/complex128 array or a CUDA torch complex tensor;
        ``normalise`` renormalises it to unit norm."""
        ptr, on_dev, is64, _keep = _buffer(psi, self.shape)
        self._check(self._lib.rotgp_set_psi(self._h, ctypes.c_void_p(ptr), on_dev, is64,
                                            int(bool(normalise))))

    def get_psi(self, out=None, fp64: bool = True):
        """Return the state as numpy (or fill ``out``: numpy or CUDA torch tensor)."""
        if out is None:
            out = np.zeros(self.shape, dtype=np.complex128 if fp64 else np.complex64)
        ptr, on_dev, is64, _keep = _buffer(out, self.shape)
        self._check(self._lib.rotgp_get_psi(self._h, ctypes.c_void_p(ptr), on_dev, is64))
        return out

    # -- propagation
    def step_imag(self, n: int = 1):
        self._check(self._lib.rotgp_step_imag(self._h, int(n)))

    def column_density(self) -> np.ndarray:
        """h_z sum_z |psi|^2 on the (N_y+1, N_x+1) plane (rotgp_column_density)."""
        out = np.zeros((self.n[1] + 1, self.n[0] + 1))
        self._check(self._lib.rotgp_column_density(
            self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0))
        return out

    def step_real(self, n: int = 1):
        self._check(self._lib.rotgp_step_real(self._h, int(n)))

    def step_schedule(self, omega, imag: bool = False):
        """len(omega) steps, step k at Omega = omega[k] (rotgp_step_schedule)."""
        om = np.ascontiguousarray(omega, dtype=np.float64)
        self._check(self._lib.rotgp_step_schedule(
            self._h, int(om.size), int(bool(imag)),
            om.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        if om.size:
            self.phys.omega = float(om[-1])

    def observables(self) -> dict:
        o = Obs()
        self._check(self._lib.rotgp_observables(self._h, ctypes.byref(o)))
        return o.as_dict()

    def sync(self):
        self._check(self._lib.rotgp_sync(self._h))

    def info(self) -> dict:
        i = SolverInfo()
        self._check(self._lib.rotgp_info(self._h, ctypes.byref(i)))
        out = {}
        for k, _ in SolverInfo._fields_:
            v = getattr(i, k)
            out[k] = list(v)[:self.dim] if isinstance(v, ctypes.Array) else v
        return out

    def tune(self, axis: int, lines_per_lane: int, chunk: int, ring: int, warps_per_block: int,
             segments: int):
        self._check(self._lib.rotgp_tune(self._h, int(axis), int(lines_per_lane), int(chunk),
                                         int(ring), int(warps_per_block), int(segments)))

    def autotune(self, steps: int = 5) -> dict:
        """Time the solver forms on this context and keep the fastest (see
        rotgp_autotune); returns the chosen form per axis."""
        ch = ctypes.c_int(0)
        self._check(self._lib.rotgp_autotune(self._h, int(steps), ctypes.byref(ch)))
        m = ch.value
        form = ["stencil" if (m >> a) & 1 else "hybrid" if (m >> (4 + a)) & 1 else "thomas"
                for a in range(self.dim)]
        if m & 8:
            form[0] = form[1] = "fused"
        return {"choice": m, "forms": form}

    def set_solver(self, axis: int, solver: str):
        """solver: "thomas", "stencil", "fused" or "hybrid" (see rotgp_set_solver)."""
        code = {"thomas": ROTGP_SOLVER_THOMAS, "stencil": ROTGP_SOLVER_STENCIL,
                "fused": ROTGP_SOLVER_FUSED, "hybrid": ROTGP_SOLVER_HYBRID}[solver]
        self._check(self._lib.rotgp_set_solver(self._h, int(axis), code))

    # -- timing
    def profile(self, on: bool = True):
        self._check(self._lib.rotgp_profile_enable(self._h, int(bool(on))))

    def profile_read(self) -> dict:
        recs = (KStat * 16)()
        cnt = ctypes.c_int(0)
        self._check(self._lib.rotgp_profile_read(self._h, recs, 16, ctypes.byref(cnt)))
        return {r.name.decode(): {"launches": r.launches, "total_ms": r.total_ms,
                                  "bytes_per_launch": r.bytes_per_launch}
                for r in recs[:cnt.value]}


class Batch:
    """Many condensates advanced together (``rotgp_batch_*``).

    specs: list of dicts with keys n, h and the physics keywords of Solver;
    precision and stream as for Solver.
    """

    def __init__(self, specs, *, precision="fp32", stream=0):
        self._lib = load()
        count = len(specs)
        grids = (Grid * count)()
        physs = (Phys * count)()
        for i, sp in enumerate(specs):
            n, h = list(sp["n"]), list(sp["h"])
            dim = len(n)
            grids[i] = Grid(dim, (ctypes.c_int * 3)(*(n + [0] * (3 - dim))),
                            (ctypes.c_double * 3)(*(h + [0.0] * (3 - dim))))
            physs[i] = Phys(sp.get("gamma", 1.0), sp.get("nu", 1.0), sp.get("lam", 1.0),
                            sp.get("g", 0.0), sp.get("omega", 0.0), sp.get("dt", 1e-3))
        handle = ctypes.c_void_p()
        rc = self._lib.rotgp_batch_create(count, grids, physs,
                                          ROTGP_FP64 if precision == "fp64" else ROTGP_FP32,
                                          ctypes.c_void_p(int(stream)), ctypes.byref(handle))
        if rc != ROTGP_OK:
            raise RotgpError(rc, self._lib.rotgp_batch_last_error(None).decode())
        self._h = handle
        self.count = count
        self.instances = []
        for i, sp in enumerate(specs):
            ch = ctypes.c_void_p()
            self._check(self._lib.rotgp_batch_context(self._h, i, ctypes.byref(ch)))
            kw = {k: sp[k] for k in ("gamma", "nu", "lam", "g", "omega", "dt") if k in sp}
            self.instances.append(Solver(sp["n"], sp["h"], precision=precision, _borrowed=ch,
                                         **kw))

    def _check(self, rc: int):
        if rc != ROTGP_OK:
            raise RotgpError(rc, self._lib.rotgp_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            for s in self.instances:
                s._h = None
            self._lib.rotgp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, steps: int = 5):
        self._check(self._lib.rotgp_batch_autotune(self._h, int(steps)))

    MODES = {"direct": 0, "graph": 1, "persistent": 2}

    def _mode(self, graph, mode):
        if mode is None:
            mode = "graph" if graph else "direct"
        return self.MODES[mode]

    def step_imag(self, n: int, graph: bool = False, mode: str | None = None):
        """mode: "direct", "graph" or "persistent" (ROTGP_BATCH_*); graph=True
        is mode "graph"."""
        self._check(self._lib.rotgp_batch_step(self._h, int(n), 1, self._mode(graph, mode)))

    def step_real(self, n: int, graph: bool = False, mode: str | None = None):
        self._check(self._lib.rotgp_batch_step(self._h, int(n), 0, self._mode(graph, mode)))

    def sync(self):
        self._check(self._lib.rotgp_batch_sync(self._h))

    def observables(self) -> list:
        out = (Obs * self.count)()
        self._check(self._lib.rotgp_batch_observables(self._h, out))
        return [o.as_dict() for o in out]

    def converge(self, rel_tol: float, check_every: int, max_steps: int, graph: bool = False,
                 mode: str | None = None):
        """Returns (steps per instance, converged flags)."""
        steps = (ctypes.c_longlong * self.count)()
        conv = (ctypes.c_int * self.count)()
        self._check(self._lib.rotgp_batch_converge(self._h, float(rel_tol), int(check_every),
                                                   int(max_steps), self._mode(graph, mode),
                                                   steps, conv))
        return list(steps), [bool(c) for c in conv]


def check_bounded_wait(stream=0) -> float:
    """Run the bounded-wait check (rotgp_check_bounded_wait); returns the
    device seconds the wait took before giving up."""
    lib = load()
    sec = ctypes.c_double(0.0)
    rc = lib.rotgp_check_bounded_wait(ctypes.c_void_p(int(stream)), ctypes.byref(sec))
    if rc != ROTGP_OK:
        raise RotgpError(rc, "the bounded wait did not give up as designed")
    return sec.value


def observables_noalloc(n, h, psi, *, gamma=1.0, nu=1.0, lam=1.0, g=0.0, omega=0.0,
                        stream=0) -> dict:
    """Observables of a CUDA tensor holding an ABI-layout wave function,
    through rotgp_observables_noalloc (no device allocation; see rotgp.h)."""
    lib = load()
    n, h = tuple(int(v) for v in n), tuple(float(v) for v in h)
    dim = len(n)
    ptr, on_dev, is64, _keep = _buffer(psi, _shape(n))
    if not on_dev:
        raise ValueError("psi must be in device memory")
    grid = Grid(dim, (ctypes.c_int * 3)(*(list(n) + [0] * (3 - dim))),
                (ctypes.c_double * 3)(*(list(h) + [0.0] * (3 - dim))))
    phys = Phys(gamma, nu, lam, g, omega, 1.0)
    o = Obs()
    rc = lib.rotgp_observables_noalloc(ctypes.byref(grid), ctypes.byref(phys),
                                       ROTGP_FP64 if is64 else ROTGP_FP32, ctypes.c_void_p(ptr),
                                       ctypes.c_void_p(int(stream)), ctypes.byref(o))
    if rc != ROTGP_OK:
        raise RotgpError(rc, lib.rotgp_last_error(None).decode())
    return o.as_dict()


def _buffer(obj, shape):
    """(pointer, on_device, is_fp64, keepalive) for numpy arrays / torch tensors."""
    if isinstance(obj, np.ndarray):
        if obj.dtype not in (np.complex64, np.complex128):
            raise TypeError("state arrays must be complex64 or complex128")
        if obj.shape != shape or not obj.flags.c_contiguous:
            raise ValueError(f"state array must be C-contiguous with shape {shape}")
        return obj.ctypes.data, 0, int(obj.dtype == np.complex128), obj
    try:
        import torch
    except ImportError as e:  # pragma: no cover
        raise TypeError("unsupported buffer type") from e
    if isinstance(obj, torch.Tensor):
        if obj.dtype not in (torch.complex64, torch.complex128):
            raise TypeError("state tensors must be complex64 or complex128")
        if tuple(obj.shape) != shape or not obj.is_contiguous():
            raise ValueError(f"state tensor must be contiguous with shape {shape}")
        return obj.data_ptr(), int(obj.is_cuda), int(obj.dtype == torch.complex128), obj
    raise TypeError("unsupported buffer type")


class WarmStart:
    """The learned warm start (``rotgp_ws_*``): proposes initial wave
    functions of 2D runs on a G x G grid of half-width L from (Omega, g, nu).
    Argument marshalling only; the network runs in the CUDA library."""

    def __init__(self, grid: int, max_batch: int = 32, stream=0):
        self._lib = load()
        self.grid, self.max_batch = int(grid), int(max_batch)
        h = ctypes.c_void_p()
        rc = self._lib.rotgp_ws_create(self.grid, self.max_batch, ctypes.c_void_p(int(stream)),
                                       ctypes.byref(h))
        if rc != ROTGP_OK:
            raise RotgpError(rc, self._lib.rotgp_ws_last_error(None).decode())
        self._h = h
        self.n_params = int(self._lib.rotgp_ws_param_count())

    def _check(self, rc):
        if rc != ROTGP_OK:
            raise RotgpError(rc, self._lib.rotgp_ws_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.rotgp_ws_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        self._check(self._lib.rotgp_ws_set_params(
            self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def get_params(self) -> np.ndarray:
        p = np.zeros(self.n_params, dtype=np.float32)
        self._check(self._lib.rotgp_ws_get_params(
            self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return p

    @staticmethod
    def _prm(prm):
        prm = np.ascontiguousarray(prm, dtype=np.float64).reshape(-1, 3)
        return prm, prm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def propose(self, prm, half_width: float, seed=None) -> np.ndarray:
        """prm: (n, 3) array of (Omega, g, nu); returns n ABI wave functions
        ((G+1) x (G+1) complex128, edges zero, not normalised); with `seed`
        multiplied by the random phase of Eq. fun drawn from that seed.  More
        than max_batch sets are proposed max_batch at a time (the phase
        depends on the point only, not on the position in the batch)."""
        prm = np.ascontiguousarray(prm, dtype=np.float64).reshape(-1, 3)
        n = prm.shape[0]
        out = np.zeros((n, self.grid + 1, self.grid + 1), dtype=np.complex128)
        for s in range(0, n, self.max_batch):
            part, pp = self._prm(prm[s:s + self.max_batch])
            dst = out[s:s + part.shape[0]]
            self._check(self._lib.rotgp_ws_propose(
                self._h, part.shape[0], pp, float(half_width), int(seed is not None),
                int(seed or 0) & 0xFFFFFFFFFFFFFFFF, ctypes.c_void_p(dst.ctypes.data), 0))
        return out

    def train_step(self, prm, half_width: float, psi, lr: float) -> float:
        """One Adam step towards the target wave functions psi (n ABI arrays,
        numpy complex128 on the host or a CUDA complex128 torch tensor)."""
        prm, pp = self._prm(prm)
        n = prm.shape[0]
        ptr, on_dev, is64, _keep = _buffer(psi, (n, self.grid + 1, self.grid + 1))
        assert is64, "targets must be complex double"
        loss = ctypes.c_double(0)
        self._check(self._lib.rotgp_ws_train_step(self._h, n, pp, float(half_width),
                                                  ctypes.c_void_p(ptr), on_dev, float(lr),
                                                  ctypes.byref(loss)))
        return loss.value

    def gradients(self, inputs, targets):
        """(loss, gradient) for given input planes [n][G][G][6] and targets
        [n][G][G][2] (float32 host arrays)."""
        x = np.ascontiguousarray(inputs, dtype=np.float32)
        t = np.ascontiguousarray(targets, dtype=np.float32)
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = ctypes.c_double(0)
        self._check(self._lib.rotgp_ws_gradients(
            self._h, x.shape[0], ctypes.c_void_p(x.ctypes.data),
            t.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(loss),
            g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return loss.value, g
