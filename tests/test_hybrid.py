"""The exact partition-method line solve (ROTGP_SOLVER_HYBRID) against the
FP64 oracle, element by element, through the C ABI.

The oracle solves every whole line with the textbook Thomas algorithm; the
hybrid form reaches the same solution with nothing truncated, so the FP64
path must match to rounding (<= 1e-10 on psi, 1e-12 relative on mu and E,
same vortex count) and the FP32 path within the FP32 tolerances (density
<= 1e-4 relative L2, mu and E <= 1e-5 relative), on ragged grids, with lines
split over clusters of 1 to 8 CTAs (including CTAs that hold no point of the
line), and on lines whose Thomas carries decay too slowly for any truncated
solver (where the chunked forms cannot run at all).
"""
import numpy as np
import pytest

import oracle
from oracle import Grid, Phys
from paper_1906_06327_gb300 import inputs
from paper_1906_06327_gb300.rotgp import Solver

from test_gpu_parity import _check_fp32, _check_fp64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()


def _run(n, h, phys, precision, nsteps, imag, hybrid_axes, clusters=None, seed=0):
    grid = Grid(n, h)
    R = inputs.random_phase_field(n[0], n[1], seed)
    ref, _ = oracle.steps(grid, phys, oracle.init_analytic(grid, 1, R), nsteps, imag)
    s = Solver(n, h, gamma=phys.gamma, nu=phys.nu, lam=phys.lam, g=phys.g, omega=phys.omega,
               dt=phys.dt, precision=precision)
    for ax in hybrid_axes:
        s.set_solver(ax, "hybrid")
        if clusters:
            s.tune(ax, 1, 8, 3, 1, clusters)
    info = s.info()
    for ax in hybrid_axes:
        assert info["hybrid_cluster"][ax] == (clusters or info["hybrid_cluster"][ax]) > 0
    s.init_analytic(1, R)
    (s.step_imag if imag else s.step_real)(nsteps)
    return s, grid, ref


CASES = [((37, 50), (0.3, 0.2)), ((64, 48), (0.25, 0.3)), ((20, 24, 18), (0.4, 0.35, 0.3)),
         ((33, 20, 17), (0.35, 0.4, 0.45))]


@pytest.mark.parametrize("n,h", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("imag", [True, False])
def test_hybrid_every_axis_matches_oracle(n, h, precision, imag):
    phys = Phys(gamma=1.0, nu=1.1, lam=1.3, g=40.0, omega=0.6, dt=2e-3)
    s, grid, ref = _run(n, h, phys, precision, 20, imag, range(len(n)))
    (_check_fp64 if precision == "fp64" else _check_fp32)(s, grid, phys, ref)


@pytest.mark.parametrize("clusters", [2, 4, 8])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_hybrid_lines_over_clusters_match_oracle(clusters, precision):
    """Lines of 200 and 96 points spread over 2..8 CTAs (8 CTAs leave the last
    ones of an x line without points)."""
    n, h = (200, 96), (0.09, 0.12)
    phys = Phys(gamma=1.0, nu=1.05, g=60.0, omega=0.7, dt=2e-3)
    for imag in (True, False):
        s, grid, ref = _run(n, h, phys, precision, 10, imag, (0, 1), clusters=clusters)
        (_check_fp64 if precision == "fp64" else _check_fp32)(s, grid, phys, ref)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_hybrid_one_axis_beside_chunked_sweeps(axis):
    n, h = (40, 36, 30), (0.3, 0.3, 0.35)
    phys = Phys(gamma=1.0, nu=1.1, lam=0.9, g=50.0, omega=0.5, dt=1e-3)
    s, grid, ref = _run(n, h, phys, "fp32", 10, True, (axis,), seed=4)
    _check_fp32(s, grid, phys, ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("imag", [False, True])
def test_lines_too_weakly_dominant_for_truncation(precision, imag):
    """Delta/h^2 = 25 (real time) or 12.5 (imaginary time): the Thomas carries
    decay by ~0.75 (~0.6) per point, so a truncated carry would need a halo of
    70 to 140 points; every sweep takes the exact solve by itself."""
    n, h = (96, 80), (0.02, 0.02)
    dt = 1e-2 if not imag else 5e-3
    phys = Phys(gamma=1.0, nu=1.05, g=20.0, omega=0.6, dt=dt)
    grid = Grid(n, h)
    R = inputs.random_phase_field(n[0], n[1], 2)
    ref, _ = oracle.steps(grid, phys, oracle.init_analytic(grid, 1, R), 10, imag)
    s = Solver(n, h, gamma=1.0, nu=1.05, g=20.0, omega=0.6, dt=dt, precision=precision)
    info = s.info()
    if precision == "fp64" or not imag:
        assert info["halo"] == 64 and all(c >= 1 for c in info["hybrid_cluster"]), info
    s.init_analytic(1, R)
    (s.step_imag if imag else s.step_real)(10)
    (_check_fp64 if precision == "fp64" else _check_fp32)(s, grid, phys, ref)
    if not imag:
        tol = 1e-12 if precision == "fp64" else 2e-5
        assert abs(s.observables()["norm"] - 1.0) < tol


@pytest.mark.slow
def test_hybrid_on_the_4096_squared_stress_grid():
    """2D 4096^2, h = 0.01 (268 MB per complex-float state): the carries decay
    by 0.31 per point (halo 19), so the complex-float plan takes the exact
    solve, with lines over clusters; two imaginary-time and two real-time
    steps against the oracle on the full grid."""
    w = inputs.WORKLOADS["2d-4096-fp32"]
    grid = Grid(w.n, w.h)
    phys = Phys(gamma=w.gamma, nu=w.nu, g=w.g, omega=w.omega, dt=w.dt)
    R = inputs.random_phase_field(w.n[0], w.n[1], 0)
    psi0 = oracle.init_analytic(grid, 1, R)
    s = Solver(w.n, w.h, gamma=w.gamma, nu=w.nu, g=w.g, omega=w.omega, dt=w.dt,
               precision="fp32")
    info = s.info()
    assert all(c >= 2 for c in info["hybrid_cluster"]), info
    s.init_analytic(1, R)
    s.step_imag(2)
    ref, _ = oracle.steps(grid, phys, psi0, 2, True)
    _check_fp32(s, grid, phys, ref)
    s.step_real(2)
    ref, _ = oracle.steps(grid, phys, ref, 2, False)
    _check_fp32(s, grid, phys, ref)
