"""FP64 CPU oracle of the rotating-GP split-step Crank-Nicolson scheme.

TEST INFRASTRUCTURE ONLY: the correctness authority for the CUDA path.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with
``paper_1906_06327_gb300`` and is never a fallback for it.

The numerics live in ``rotgp_oracle.c`` (plain C99 complex double, single
thread); this module compiles it with gcc and wraps it with ctypes.  Arrays
are numpy ``complex128`` holding all (N+1)^d grid points, edges included, x
fastest (shape ``(N_z+1, N_y+1, N_x+1)`` in 3D, ``(N_y+1, N_x+1)`` in 2D), as
the paper's programs store them (Sec. 3, "(NX+1) x (NY+1) points").

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(the real-part energy and chemical potential at g != 0 through their
identity with the complex forms on states e^{i theta} f, f real).
``warmstart_ref`` (the FP64 reference of the learned start's network) is
pinned by ``tests/test_warmstart_ref.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rotgp_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.orc_thomas_d.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp]
        lib.orc_substep.argtypes = [ctypes.c_int, ip, dp, dp, ctypes.c_int,
                                    ctypes.c_int, dp]
        lib.orc_steps.argtypes = [ctypes.c_int, ip, dp, dp, ctypes.c_int,
                                  ctypes.c_longlong, dp, dp]
        lib.orc_norm.argtypes = [ctypes.c_int, ip, dp, dp]
        lib.orc_norm.restype = ctypes.c_double
        lib.orc_init_analytic.argtypes = [ctypes.c_int, ip, dp, ctypes.c_int, dp,
                                          ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, dp]
        lib.orc_observables.argtypes = [ctypes.c_int, ip, dp, dp, dp, dp]
        lib.orc_vortex_count.argtypes = [ctypes.c_int, ip, dp, dp, ctypes.c_int]
        _lib = lib
        return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass(frozen=True)
class Grid:
    """n = numbers of intervals per axis (points are n+1), h = spacings."""
    n: tuple
    h: tuple

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def shape(self) -> tuple:
        return tuple(int(v) + 1 for v in reversed(self.n))

    def coords(self, axis: int) -> np.ndarray:
        N, h = self.n[axis], self.h[axis]
        return -0.5 * N * h + np.arange(N + 1) * h

    def _c(self):
        n = (ctypes.c_int * 3)(*(list(self.n) + [0] * (3 - self.dim)))
        h = (ctypes.c_double * 3)(*(list(self.h) + [0.0] * (3 - self.dim)))
        return n, h


@dataclass(frozen=True)
class Phys:
    gamma: float = 1.0
    nu: float = 1.0
    lam: float = 1.0
    g: float = 0.0
    omega: float = 0.0
    dt: float = 1e-3

    def _c(self):
        return (ctypes.c_double * 6)(self.gamma, self.nu, self.lam, self.g,
                                     self.omega, self.dt)


OBS_KEYS = ("norm", "mu", "energy", "mu_c", "energy_c", "rms_x", "rms_y",
            "rms_z", "rms_r", "max_density", "mu4", "energy4")


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def _as_psi(grid: Grid, psi: np.ndarray) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    if psi.shape != grid.shape:
        raise ValueError(f"psi shape {psi.shape} != grid shape {grid.shape}")
    return psi


def thomas(am: complex, a0: complex, ap: complex, b: np.ndarray) -> np.ndarray:
    """Solve the constant-coefficient tridiagonal system by the Thomas algorithm."""
    lib = _load()
    b = np.ascontiguousarray(b, dtype=np.complex128)
    x = np.zeros_like(b)
    c = [np.array([v.real, v.imag]) for v in (complex(am), complex(a0), complex(ap))]
    _check(lib.orc_thomas_d(len(b), _dptr(c[0]), _dptr(c[1]), _dptr(c[2]),
                            _dptr(b), _dptr(x)), "thomas")
    return x


def substep(grid: Grid, phys: Phys, psi: np.ndarray, which: int, imag: bool) -> np.ndarray:
    """which = 0 (H1), 1 (x-sweep), 2 (y-sweep), 3 (z-sweep); returns a new array."""
    lib = _load()
    out = _as_psi(grid, psi).copy()
    n, h = grid._c()
    _check(lib.orc_substep(grid.dim, n, h, phys._c(), int(imag), which, _dptr(out)),
           "substep")
    return out


def steps(grid: Grid, phys: Phys, psi: np.ndarray, nsteps: int, imag: bool):
    """Run nsteps full split steps; returns (new psi, last discrete norm)."""
    lib = _load()
    out = _as_psi(grid, psi).copy()
    n, h = grid._c()
    last = ctypes.c_double(0.0)
    _check(lib.orc_steps(grid.dim, n, h, phys._c(), int(imag), int(nsteps),
                         _dptr(out), ctypes.byref(last)), "steps")
    return out, last.value


def norm(grid: Grid, psi: np.ndarray) -> float:
    lib = _load()
    n, h = grid._c()
    return lib.orc_norm(grid.dim, n, h, _dptr(_as_psi(grid, psi)))


def init_analytic(grid: Grid, function: int = 1, R: np.ndarray | None = None,
                  d_xy: float = 1.0, d_z: float = 1.0, normalize: bool = True) -> np.ndarray:
    """Initial state of Eq. fun; R is the (N_y+1, N_x+1) random field in [0,1) or None."""
    lib = _load()
    out = np.zeros(grid.shape, dtype=np.complex128)
    n, h = grid._c()
    Rp = None
    if R is not None:
        R = np.ascontiguousarray(R, dtype=np.float64)
        if R.shape != (grid.n[1] + 1, grid.n[0] + 1):
            raise ValueError("R must have shape (N_y+1, N_x+1)")
        Rp = _dptr(R)
    _check(lib.orc_init_analytic(grid.dim, n, h, int(function), Rp, float(d_xy),
                                 float(d_z), int(normalize), _dptr(out)),
           "init_analytic")
    return out


def observables(grid: Grid, phys: Phys, psi: np.ndarray) -> dict:
    lib = _load()
    out = np.zeros(len(OBS_KEYS))
    n, h = grid._c()
    _check(lib.orc_observables(grid.dim, n, h, phys._c(), _dptr(_as_psi(grid, psi)),
                               _dptr(out)), "observables")
    return dict(zip(OBS_KEYS, out.tolist()))


def vortex_count(grid: Grid, psi: np.ndarray, fp32_decision: bool = False) -> int:
    lib = _load()
    n, h = grid._c()
    c = lib.orc_vortex_count(grid.dim, n, h, _dptr(_as_psi(grid, psi)),
                             int(fp32_decision))
    if c < 0:
        raise RuntimeError("oracle vortex_count failed")
    return int(c)
