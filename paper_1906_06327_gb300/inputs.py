"""Seeded synthetic inputs and workload definitions.

This module holds no arithmetic of the method itself: it only draws the
random numbers the initial state consumes and names the workloads.  Both the
CUDA path and the CPU oracle receive what it produces as plain inputs.

Random phase field R(x, y) of Eq. fun
    R_n = (SplitMix64 output n of the stream seeded with ``seed``) >> 11,
    scaled by 2^-53 into [0, 1), for n = j (N_x + 1) + i on the paper's
    (N_x + 1) x (N_y + 1) plane (x fastest).  SplitMix64 is the generator of
    Steele, Lea and Flood, "Fast splittable pseudorandom number generators"
    (OOPSLA 2014): state s_n = seed + (n + 1) * 0x9E3779B97F4A7C15, output
    z = s_n; z = (z ^ z>>30) * 0xBF58476D1CE4E5B9; z = (z ^ z>>27) *
    0x94D049BB133111EB; z ^ z>>31 (all mod 2^64).  Being counter based, any
    element can be regenerated independently.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of the SplitMix64 stream seeded with seed."""
    with np.errstate(over="ignore"):
        n = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + n * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def random_phase_field(n_x: int, n_y: int, seed: int) -> np.ndarray:
    """R in [0,1) on the (n_y+1, n_x+1) plane of a grid with n intervals."""
    z = splitmix64(seed, (n_x + 1) * (n_y + 1))
    r = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return r.reshape(n_y + 1, n_x + 1)


@dataclass(frozen=True)
class Workload:
    """One solver configuration: grid (intervals, spacings) and physics."""
    name: str
    n: tuple
    h: tuple
    gamma: float
    nu: float
    lam: float
    g: float
    omega: float
    dt: float
    imag_steps: int
    real_steps: int = 0
    real_dt: float = 1e-4
    seed: int = 0
    precision: str = "fp32"
    extra: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return len(self.n)

    @property
    def sites(self) -> int:
        s = 1
        for v in self.n:
            s *= int(v)
        return s


# 2D, imaginary time, FP64: 128^2 intervals, dx = dy = 0.1 (domain +-6.4),
# gamma = nu = 1, g = 100, Omega = 0.5, dt = 1e-3, 1000 steps, seed 0.
WL_2D_128_FP64 = Workload("2d-128-imag-fp64", (128, 128), (0.1, 0.1), 1.0, 1.0,
                          1.0, 100.0, 0.5, 1e-3, 1000, precision="fp64")

# 2D, FP32 bulk: 512^2, dx = 0.05, gamma = 1, nu = 1.05, g = 1000, Omega = 0.9,
# imaginary dt = 2.5e-4 x 40000, then real dt = 1e-4 x 20000 (Omega ramped to 0.8).
WL_2D_512_FP32 = Workload("2d-512-fp32", (512, 512), (0.05, 0.05), 1.0, 1.05,
                          1.0, 1000.0, 0.9, 2.5e-4, 40000, 20000, 1e-4,
                          extra={"omega_ramp_to": 0.8})

# 3D, complex FP32: 256 x 256 x 128, dx = dy = 0.08, dz = 0.1, gamma = nu = 1,
# lambda = 0.5, g = 3000, Omega = 0.85, imaginary dt = 2e-4 x 20000, then
# 5000 real-time steps (dt 1e-4).
WL_3D_256_FP32 = Workload("3d-256x256x128-fp32", (256, 256, 128), (0.08, 0.08, 0.1),
                          1.0, 1.0, 0.5, 3000.0, 0.85, 2e-4, 20000, 5000, 1e-4)

# A larger-than-L2 2D shape with the 512^2 physics: 4096^2, dx = 0.01.
WL_2D_4096_FP32 = Workload("2d-4096-fp32", (4096, 4096), (0.01, 0.01), 1.0, 1.05,
                           1.0, 1000.0, 0.9, 2.5e-4, 0)

# A larger-than-L2 3D shape with the 256 x 256 x 128 physics: 512 x 512 x 128
# (268 MB per complex-float state, twice the L2).
WL_3D_512_FP32 = Workload("3d-512x512x128-fp32", (512, 512, 128), (0.08, 0.08, 0.1),
                          1.0, 1.0, 0.5, 3000.0, 0.85, 2e-4, 0)

WORKLOADS = {w.name: w for w in (WL_2D_128_FP64, WL_2D_512_FP32, WL_3D_256_FP32,
                                 WL_2D_4096_FP32, WL_3D_512_FP32)}


def batch_specs(count: int = 64, seed: int = 0, dt: float = 5e-4) -> list:
    """Instances of the batched 2D workload, seeded: N drawn from
    {128, 256, 384, 512}, Omega ~ U[0.3, 0.95], g ~ U[100, 2000],
    nu ~ U[1.0, 1.1], gamma = 1; the domain half-width is 1.3 R_TF + 2 with
    the Thomas-Fermi radius R_TF = (4 g / (pi (1 - Omega^2)))^(1/4), so that
    h = 2 (1.3 R_TF + 2) / N; dt = 5e-4 for every instance.  Uniform numbers
    come from SplitMix64(seed), five per instance."""
    u = splitmix64(seed, 5 * count).astype(np.float64) / 2.0**64
    out = []
    for i in range(count):
        r = u[5 * i:5 * i + 5]
        n = (128, 256, 384, 512)[min(3, int(r[0] * 4))]
        omega = 0.3 + 0.65 * r[1]
        g = 100.0 + 1900.0 * r[2]
        nu = 1.0 + 0.1 * r[3]
        r_tf = (4.0 * g / (np.pi * (1.0 - omega * omega))) ** 0.25
        h = 2.0 * (1.3 * r_tf + 2.0) / n
        out.append(dict(n=(n, n), h=(float(h), float(h)), gamma=1.0, nu=float(nu), g=float(g),
                        omega=float(omega), dt=dt, seed=int(r[4] * 2**31)))
    return out


def warmstart_params(count: int, seed: int, omega=(0.7, 0.9), g=(200.0, 800.0),
                     nu=(1.0, 1.1)) -> np.ndarray:
    """(count, 3) parameter sets (Omega, g, nu) of the learned-warm-start
    workload, uniform in the given ranges; three SplitMix64(seed) numbers per
    set."""
    u = splitmix64(seed, 3 * count).astype(np.float64) / 2.0**64
    u = u.reshape(count, 3)
    return np.stack([omega[0] + (omega[1] - omega[0]) * u[:, 0],
                     g[0] + (g[1] - g[0]) * u[:, 1],
                     nu[0] + (nu[1] - nu[0]) * u[:, 2]], axis=1)
