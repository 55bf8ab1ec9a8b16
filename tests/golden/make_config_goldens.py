"""Write the oracle's expected values for the full-length runs of the 512^2
and 256 x 256 x 128 workloads (FP64 CPU oracle only; nothing here touches
the CUDA library).

512^2 (h = 0.05, gamma = 1, nu = 1.05, g = 1000, Omega = 0.9): 40,000
imaginary-time steps of Delta = 2.5e-4 from the seed-0 one-vortex start of
Eq. fun, then 20,000 real-time steps of Delta = 1e-4 with Omega lowered
linearly, Omega_k = 0.9 - 0.1 k / 20000 for step k = 0 .. 19999 (held fixed
within a step), as Sec. 3 runs real-time dynamics from an imaginary-time
state.  Stored: the observables after 10,000, 20,000 and 40,000 imaginary
steps and after the ramp, and |psi|^2 on every 4th grid point after each
part.

256 x 256 x 128 (h = 0.08, 0.08, 0.1, lambda = 0.5, g = 3000, Omega = 0.85,
Delta = 2e-4): 200 imaginary-time steps from the seed-0 start; stored: the
observables and |psi|^2 on every 4th point in x and y and every 8th in z.

Run:  python tests/golden/make_config_goldens.py [512|3d|all]   (~25 min for 512)
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1906_06327_gb300 import inputs  # noqa: E402

KEYS = oracle.OBS_KEYS


def _obs(grid, phys, psi):
    o = oracle.observables(grid, phys, psi)
    return np.array([o[k] for k in KEYS] + [oracle.vortex_count(grid, psi)], dtype=np.float64)


def make_512():
    w = inputs.WORKLOADS["2d-512-fp32"]
    grid = oracle.Grid(w.n, w.h)
    phys = oracle.Phys(gamma=w.gamma, nu=w.nu, g=w.g, omega=w.omega, dt=w.dt)
    psi = oracle.init_analytic(grid, 1, inputs.random_phase_field(w.n[0], w.n[1], w.seed))
    obs, marks = [], []
    t0 = time.time()
    for upto in (10000, 20000, 40000):
        psi, _ = oracle.steps(grid, phys, psi, upto - (marks[-1] if marks else 0), True)
        marks.append(upto)
        obs.append(_obs(grid, phys, psi))
        print(f"imag {upto}: mu {obs[-1][1]:.8f} ({time.time() - t0:.0f} s)", flush=True)
    dens_imag = (np.abs(psi) ** 2)[::4, ::4].copy()
    nreal, om0, om1 = w.real_steps, w.omega, w.extra["omega_ramp_to"]
    for k in range(nreal):
        pk = oracle.Phys(gamma=w.gamma, nu=w.nu, g=w.g, omega=om0 + (om1 - om0) * k / nreal,
                         dt=w.real_dt)
        psi, _ = oracle.steps(grid, pk, psi, 1, False)
    pend = oracle.Phys(gamma=w.gamma, nu=w.nu, g=w.g,
                       omega=om0 + (om1 - om0) * (nreal - 1) / nreal, dt=w.real_dt)
    obs.append(_obs(grid, pend, psi))
    print(f"real {nreal}: norm {obs[-1][0]:.12f} ({time.time() - t0:.0f} s)", flush=True)
    np.savez_compressed(os.path.join(HERE, "config_512_oracle.npz"), keys=np.array(KEYS + ("vortices",)),
                        marks=np.array(marks + [nreal]), obs=np.array(obs),
                        dens_imag=dens_imag, dens_real=(np.abs(psi) ** 2)[::4, ::4].copy(),
                        stride=np.array([4, 4]))


def make_3d():
    w = inputs.WORKLOADS["3d-256x256x128-fp32"]
    grid = oracle.Grid(w.n, w.h)
    phys = oracle.Phys(gamma=w.gamma, nu=w.nu, lam=w.lam, g=w.g, omega=w.omega, dt=w.dt)
    psi = oracle.init_analytic(grid, 1, inputs.random_phase_field(w.n[0], w.n[1], w.seed))
    t0 = time.time()
    psi, _ = oracle.steps(grid, phys, psi, 200, True)
    ob = _obs(grid, phys, psi)
    print(f"3d 200: mu {ob[1]:.8f} ({time.time() - t0:.0f} s)", flush=True)
    np.savez_compressed(os.path.join(HERE, "config_3d_200_oracle.npz"),
                        keys=np.array(KEYS + ("vortices",)), steps=np.array([200]),
                        obs=ob[None, :],
                        dens=(np.abs(psi) ** 2)[::8, ::4, ::4].astype(np.float32),
                        stride=np.array([4, 4, 8]))


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "all"
    if what in ("3d", "all"):
        make_3d()
    if what in ("512", "all"):
        make_512()
