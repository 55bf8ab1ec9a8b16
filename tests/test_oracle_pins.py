"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test would fail under a plausible mistake in the oracle: a dropped term,
a wrong sign of the rotation coefficient in either sweep, a transposed axis,
a wrong quadrature weight or a broken line solve.
"""
import os

import numpy as np
import pytest
from scipy.linalg import eigh_tridiagonal

import oracle
from oracle import Grid, Phys
from paper_1906_06327_gb300 import inputs

from dense_ops import DenseOps

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- inputs
def test_splitmix64_reference_vectors():
    """The counter-based generator reproduces its published reference outputs."""
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    for row in rows:
        seed, want = int(row[0]), [int(v, 16) for v in row[1:]]
        got = [int(v) for v in inputs.splitmix64(seed, len(want))]
        assert got == want
        # counter based: any window regenerates the same numbers
        assert [int(v) for v in inputs.splitmix64(seed, 2, offset=1)] == want[1:3]


def test_random_phase_field_range():
    R = inputs.random_phase_field(64, 32, 0)
    assert R.shape == (33, 65)
    assert R.min() >= 0.0 and R.max() < 1.0
    assert abs(R.mean() - 0.5) < 0.02


# ---------------------------------------------------------------- line solve
@pytest.mark.parametrize("m", [1, 2, 3, 7, 31, 64])
def test_thomas_matches_dense_solve(m):
    rng = np.random.default_rng(m)
    for _ in range(3):
        am, ap = rng.normal(size=2) + 1j * rng.normal(size=2)
        a0 = 3.0 + abs(am) + abs(ap) + 1j * rng.normal()
        b = rng.normal(size=m) + 1j * rng.normal(size=m)
        A = (np.diag(np.full(m, a0)) + np.diag(np.full(m - 1, am), -1)
             + np.diag(np.full(m - 1, ap), 1))
        want = np.linalg.solve(A, b)
        got = oracle.thomas(am, a0, ap, b)
        assert np.max(np.abs(got - want)) < 1e-13 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("imag", [False, True])
def test_x_and_y_sweeps_toeplitz_eigenpairs(imag):
    """One CN sweep maps the closed-form Toeplitz eigenvector
    v_i = rho^i sin(i k pi / N), rho^2 = A-/A+, to
    [(1 - 2 kappa) - 2 A+ rho cos(k pi/N)] / [A0 + 2 A+ rho cos(k pi/N)] v,
    with the coefficients of Eq. eq5 (and i Delta -> Delta in imaginary time)."""
    nx, ny, hx, hy = 24, 20, 0.3, 0.25
    dt, omega = 2e-2, 0.7
    grid = Grid((nx, ny), (hx, hy))
    phys = Phys(gamma=1.0, nu=1.2, g=0.0, omega=omega, dt=dt)
    idt = dt if imag else 1j * dt
    for axis, (N, h, n_other) in enumerate([(nx, hx, ny), (ny, hy, nx)]):
        k = 3
        theta = k * np.pi / N
        other = Grid((nx, ny), (hx, hy)).coords(1 - axis)
        psi = np.zeros(grid.shape, dtype=np.complex128)
        lam = np.zeros(n_other + 1, dtype=np.complex128)
        for q in range(1, n_other):
            rot = omega * other[q] if axis == 0 else -omega * other[q]
            am = -(idt / (4 * h)) * (1 / h - 1j * rot)
            ap = -(idt / (4 * h)) * (1 / h + 1j * rot)
            a0 = 1 + idt / (2 * h * h)
            kappa = idt / (4 * h * h)
            rho = np.sqrt(am / ap)
            i = np.arange(N + 1)
            v = rho ** i * np.sin(i * theta) * (1.0 + 0.1 * q)
            lam[q] = ((1 - 2 * kappa) - 2 * ap * rho * np.cos(theta)) / (
                a0 + 2 * ap * rho * np.cos(theta))
            if axis == 0:
                psi[q, :] = v
            else:
                psi[:, q] = v
        out = oracle.substep(grid, phys, psi, 1 + axis, imag)
        want = psi * (lam[:, None] if axis == 0 else lam[None, :])
        assert np.max(np.abs(out - want)) < 1e-13 * np.max(np.abs(psi))


# ---------------------------------------------------------------- full step
@pytest.mark.parametrize("imag", [False, True])
@pytest.mark.parametrize("shape", [((8, 8), (0.7, 0.6)), ((6, 6, 6), (0.9, 0.8, 0.7))])
def test_full_step_matches_dense_operator_brute_force(imag, shape):
    """Oracle's split step equals H1 then dense CN solves of the operators of
    Eqs. eq2/eq3 (+ z), built independently of the coefficients of Eq. eq5."""
    n, h = shape
    grid = Grid(n, h)
    phys = Phys(gamma=1.0, nu=1.3, lam=0.8, g=7.0, omega=0.6, dt=0.05)
    ops = DenseOps(n, h, phys.gamma, phys.nu, phys.lam, phys.g, phys.omega)
    R = inputs.random_phase_field(n[0], n[1], 5)
    psi0 = oracle.init_analytic(grid, 1, R, 1.0, 1.0)
    got, _ = oracle.steps(grid, phys, psi0, 3, imag)
    v = ops.interior(psi0)
    for _ in range(3):
        v = ops.step(v, phys.dt, imag)
    want = ops.full(v)
    assert np.max(np.abs(got - want)) < 1e-12


def test_h1_substep_closed_form():
    n, h = (10, 12), (0.5, 0.4)
    grid = Grid(n, h)
    phys = Phys(gamma=1.1, nu=0.9, g=30.0, dt=0.01)
    psi = oracle.init_analytic(grid, 1, inputs.random_phase_field(*n, 1))
    x, y = grid.coords(0)[None, :], grid.coords(1)[:, None]
    V = 0.5 * (phys.gamma ** 2 * x ** 2 + phys.nu ** 2 * y ** 2)
    dens = np.abs(psi) ** 2
    re = oracle.substep(grid, phys, psi, 0, False)
    im = oracle.substep(grid, phys, psi, 0, True)
    # real time: modulus unchanged, phase advanced by -Delta (V + g|psi|^2)
    assert np.max(np.abs(np.abs(re) - np.abs(psi))) < 1e-15
    mask = dens > 1e-20
    dphi = np.angle(re[mask] / psi[mask])
    assert np.max(np.abs(dphi + phys.dt * (V + phys.g * dens)[mask])) < 1e-12
    # imaginary time: real positive factor exp(-Delta (V + g|psi|^2))
    ratio = im[mask] / psi[mask]
    assert np.max(np.abs(ratio.imag)) < 1e-15
    assert np.max(np.abs(np.log(ratio.real) + phys.dt * (V + phys.g * dens)[mask])) < 1e-12


# ---------------------------------------------------------------- physics
def _exact_1d_ground(N, h, w):
    """Smallest eigenvalue of -(1/2) D2 + w^2 x^2 / 2 on the interior points."""
    x = -0.5 * N * h + np.arange(1, N) * h
    d = 1.0 / h ** 2 + 0.5 * w ** 2 * x ** 2
    e = np.full(N - 2, -0.5 / h ** 2)
    return eigh_tridiagonal(d, e, eigvals_only=True, select="i", select_range=(0, 0))[0]


def test_harmonic_ground_energy_2d():
    """g = 0, Omega = 0: E = mu -> (gamma + nu)/2 with O(h^2) discretisation
    error; the imaginary-time fixed point equals the discrete ground energy."""
    gamma, nu = 1.0, 1.5
    errs = []
    for N, h in [(32, 0.4), (64, 0.2)]:
        grid = Grid((N, N), (h, h))
        phys = Phys(gamma=gamma, nu=nu, g=0.0, omega=0.0, dt=5e-3)
        psi = oracle.init_analytic(grid, 0, inputs.random_phase_field(N, N, 2))
        psi, _ = oracle.steps(grid, phys, psi, 4000, True)
        ob = oracle.observables(grid, phys, psi)
        e_disc = _exact_1d_ground(N, h, gamma) + _exact_1d_ground(N, h, nu)
        # Lie splitting of CN substeps: the fixed point's energy is off the
        # discrete ground energy by O(Delta^2) (first-order eigenvector error)
        assert abs(ob["energy_c"] - e_disc) < 1e-5
        assert abs(ob["mu_c"] - ob["energy_c"]) < 1e-12
        assert abs(ob["norm"] - 1.0) < 1e-13
        errs.append(abs(ob["energy_c"] - (gamma + nu) / 2))
        # rms of the Gaussian ground state: <x^2> = 1/(2 gamma)
        assert abs(ob["rms_x"] - np.sqrt(0.5 / gamma)) < 0.01
        assert abs(ob["rms_y"] - np.sqrt(0.5 / nu)) < 0.01
    assert errs[1] < 5e-3
    assert 3.0 < errs[0] / errs[1] < 5.0  # second order in h


def test_imaginary_time_fixed_point_error_is_second_order_in_dt():
    N, h = 32, 0.4
    grid = Grid((N, N), (h, h))
    e_disc = _exact_1d_ground(N, h, 1.0) + _exact_1d_ground(N, h, 1.5)
    errs = []
    for dt in (1e-2, 5e-3):
        phys = Phys(gamma=1.0, nu=1.5, g=0.0, omega=0.0, dt=dt)
        psi = oracle.init_analytic(grid, 0, inputs.random_phase_field(N, N, 2))
        psi, _ = oracle.steps(grid, phys, psi, int(20 / dt), True)
        errs.append(oracle.observables(grid, phys, psi)["energy_c"] - e_disc)
    assert errs[0] > 0 and errs[1] > 0
    assert 3.8 < errs[0] / errs[1] < 4.2


def test_harmonic_ground_energy_3d():
    """g = 0, Omega = 0: E -> (gamma + nu + lambda)/2 in 3D (pins the z sweep)."""
    gamma, nu, lam = 1.0, 1.3, 2.0
    n, h = (20, 20, 20), (0.5, 0.5, 0.4)
    grid = Grid(n, h)
    phys = Phys(gamma=gamma, nu=nu, lam=lam, g=0.0, omega=0.0, dt=5e-3)
    psi = oracle.init_analytic(grid, 0, inputs.random_phase_field(20, 20, 3))
    psi, _ = oracle.steps(grid, phys, psi, 3000, True)
    ob = oracle.observables(grid, phys, psi)
    e_disc = (_exact_1d_ground(20, 0.5, gamma) + _exact_1d_ground(20, 0.5, nu)
              + _exact_1d_ground(20, 0.4, lam))
    assert abs(ob["energy_c"] - e_disc) < phys.dt ** 2  # O(Delta^2), see 2D
    assert abs(ob["energy_c"] - (gamma + nu + lam) / 2) < 0.05


def test_rotating_ground_state_matches_dense_eigensolver():
    """Anisotropic trap with rotation (not separable): the imaginary-time fixed
    point's energy equals the smallest eigenvalue of the dense discrete
    H = -lap/2 + V - Omega L_z (Eq. e2d at g = 0) up to O(Delta^2)."""
    N, h = 20, 0.6
    phys = Phys(gamma=1.0, nu=1.3, g=0.0, omega=0.5, dt=5e-3)
    grid = Grid((N, N), (h, h))
    ops = DenseOps((N, N), (h, h), phys.gamma, phys.nu, 1.0, 0.0, phys.omega)
    lam_min = np.linalg.eigvalsh(ops.Hlin)[0]
    psi = oracle.init_analytic(grid, 0, inputs.random_phase_field(N, N, 4))
    psi, _ = oracle.steps(grid, phys, psi, 8000, True)
    ob = oracle.observables(grid, phys, psi)
    assert abs(ob["energy_c"] - lam_min) < 2e-5
    # Rayleigh quotient of the dense operator for the same state
    v = ops.interior(psi)
    rq = np.real(np.vdot(v, ops.Hlin @ v) / np.vdot(v, v))
    assert abs(ob["energy_c"] - rq) < 1e-12


def test_one_vortex_energy_two_minus_omega():
    """(x + i y) exp(-r^2/2) is an L_z = +1 eigenstate of the isotropic trap:
    E = mu = 2 - Omega at g = 0 (Eqs. e2d and e2dr), to O(h^2)."""
    N, h, omega = 128, 0.1, 0.5
    grid = Grid((N, N), (h, h))
    phys = Phys(gamma=1.0, nu=1.0, g=0.0, omega=omega, dt=1e-3)
    psi = oracle.init_analytic(grid, 1, None)
    ob = oracle.observables(grid, phys, psi)
    for key in ("energy", "mu", "energy_c", "mu_c"):
        assert abs(ob[key] - (2 - omega)) < 2e-3, key
    assert abs(ob["energy"] - ob["energy_c"]) < 1e-9


def test_imaginary_time_selects_positive_circulation():
    """From the real state x exp(-r^2/2) (equal parts m = +1 and m = -1), at
    g = 0 and Omega > 0 imaginary time must converge to the m = +1 vortex with
    E = 2 - Omega; a wrong sign of the rotation term in either sweep would pick
    m = -1 (E = 2 + Omega) or no eigenstate at all."""
    N, h, omega = 64, 0.2, 0.5
    grid = Grid((N, N), (h, h))
    phys = Phys(gamma=1.0, nu=1.0, g=0.0, omega=omega, dt=2e-3)
    psi = oracle.init_analytic(grid, 1, None).real.astype(np.complex128)
    psi, _ = oracle.steps(grid, phys, psi, 5000, True)
    ob = oracle.observables(grid, phys, psi)
    assert abs(ob["energy_c"] - (2 - omega)) < 5e-3
    ob0 = oracle.observables(grid, Phys(gamma=1.0, nu=1.0, g=0.0, omega=0.0), psi)
    lz = (ob0["energy_c"] - ob["energy_c"]) / omega
    assert abs(lz - 1.0) < 0.02  # discrete L_z: O(h^2) off the integer
    # the core of this symmetric state sits exactly on the centre node (psi = 0
    # there), which the plaquette count cannot see; shift by half a cell
    assert oracle.vortex_count(grid, np.roll(psi, 1, axis=0)) == 1


def test_real_time_conserves_norm_and_energy():
    """Each real-time substep is unitary (H1 is a phase; CN of a Hermitian
    discrete H2/H3 is a Cayley transform): the discrete norm is conserved to
    rounding, and the energy only fluctuates at O(Delta)."""
    N, h = 48, 0.25
    grid = Grid((N, N), (h, h))
    phys = Phys(gamma=1.0, nu=1.1, g=40.0, omega=0.6, dt=1e-3)
    psi0 = oracle.init_analytic(grid, 1, None)
    psi0 = np.roll(psi0, 3, axis=1)  # displaced: a non-stationary start
    psi0[:, :3] = 0
    psi0 /= np.sqrt(oracle.norm(grid, psi0))
    e0 = oracle.observables(grid, phys, psi0)["energy_c"]
    psi, nrm = oracle.steps(grid, phys, psi0, 2000, False)
    ob = oracle.observables(grid, phys, psi)
    # rounding only: ~1e-15 per step (a non-unitary substep would drift at
    # O(Delta) = 1e-3 per unit time)
    assert abs(nrm - 1.0) < 2e-11
    assert abs(ob["norm"] - 1.0) < 2e-11
    assert abs(ob["energy_c"] - e0) / e0 < 2e-3


def test_real_time_norm_3d():
    n, h = (16, 16, 12), (0.5, 0.5, 0.4)
    grid = Grid(n, h)
    phys = Phys(gamma=1.0, nu=1.0, lam=1.5, g=20.0, omega=0.7, dt=2e-3)
    psi0 = oracle.init_analytic(grid, 1, inputs.random_phase_field(16, 16, 9))
    psi, nrm = oracle.steps(grid, phys, psi0, 300, False)
    assert abs(nrm - 1.0) < 1e-12 * 300 / 100


def test_omega_zero_reduces_to_non_rotating():
    """Omega = 0: a real state stays exactly real in imaginary time, and at
    g = 0 a product state f(x) g(y) stays a product (the sweeps decouple)."""
    N, h = 32, 0.3
    grid = Grid((N, N), (h, h))
    phys = Phys(gamma=1.0, nu=1.4, g=50.0, omega=0.0, dt=2e-3)
    psi0 = oracle.init_analytic(grid, 0, None)
    psi, _ = oracle.steps(grid, phys, psi0, 200, True)
    assert np.max(np.abs(psi.imag)) == 0.0
    phys0 = Phys(gamma=1.0, nu=1.4, g=0.0, omega=0.0, dt=2e-3)
    x = grid.coords(0)
    f = np.exp(-(x - 0.7) ** 2) * (1 + 0.3 * x)
    gy = np.exp(-(x + 0.4) ** 2 / 2) * (1 + 1j * 0.2 * x)
    prod = (gy[:, None] * f[None, :]).astype(np.complex128)
    prod[0, :] = prod[-1, :] = 0
    prod[:, 0] = prod[:, -1] = 0
    out, _ = oracle.steps(grid, phys0, prod, 50, True)
    s = np.linalg.svd(out, compute_uv=False)
    assert s[1] / s[0] < 1e-13


# ---------------------------------------------------------------- observables
def test_energy_forms_agree_with_dense_rayleigh_quotient():
    """E_c is the Rayleigh quotient of the discrete Hamiltonian at g = 0 for any
    state; for a real state the real-part form (Eq. e2dr) gives the same."""
    N, h = (12, 10), (0.5, 0.6)
    grid = Grid(N, h)
    phys = Phys(gamma=1.0, nu=1.2, g=0.0, omega=0.4)
    ops = DenseOps(N, h, 1.0, 1.2, 1.0, 0.0, 0.4)
    psi = oracle.init_analytic(grid, 1, inputs.random_phase_field(*N, 8))
    v = ops.interior(psi)
    rq = np.real(np.vdot(v, ops.Hlin @ v) / np.vdot(v, v))
    ob = oracle.observables(grid, phys, psi)
    assert abs(ob["energy_c"] - rq) < 1e-12
    assert abs(ob["mu_c"] - rq) < 1e-12
    real_psi = psi.real.astype(np.complex128)
    ob_r = oracle.observables(grid, phys, real_psi)
    vr = ops.interior(real_psi)
    rq_r = np.real(np.vdot(vr, ops.Hlin @ vr) / np.vdot(vr, vr))
    assert abs(ob_r["energy"] - rq_r) < 1e-12
    # global phase -i: the guard rotates back and gives the same value
    ob_rot = oracle.observables(grid, phys, -1j * real_psi)
    assert abs(ob_rot["energy"] - rq_r) < 1e-12


def test_real_part_mu_equals_complex_mu_on_a_stationary_state():
    """On a stationary state the real-part equation (Eqs. e2dr/e3dr: the real
    part of mu psi = H psi, with the rotation coupling Omega (y D_x - x D_y)
    psi_I and the nonlinear g |psi|^2 psi_R) and the complex Rayleigh
    quotient give the same mu.  The imaginary-time fixed point of the split
    step (H1, x, y: a first-order splitting, Sec. 2) is stationary up to
    O(Delta), so the two forms must approach each other linearly in Delta on
    a rotating, interacting, anisotropic vortex state."""
    N, h = (24, 24), (0.35, 0.35)
    grid = Grid(N, h)
    diffs = []
    for dt in (4e-3, 2e-3):
        phys = Phys(gamma=1.0, nu=1.2, g=15.0, omega=0.5, dt=dt)
        psi = oracle.init_analytic(grid, 1, inputs.random_phase_field(*N, 3))
        psi, _ = oracle.steps(grid, phys, psi, int(40 / dt), True)
        ob = oracle.observables(grid, phys, psi)
        diffs.append(abs(ob["mu"] - ob["mu_c"]))
    assert diffs[0] < 1e-4 * 2.65
    assert 1.7 < diffs[0] / diffs[1] < 2.3, diffs


def test_nonlinear_energy_term_closed_form():
    """The g terms of E_c and mu_c are g/2 and g times h^d sum |psi|^4 (unit norm)."""
    N, h = (16, 16), (0.4, 0.4)
    grid = Grid(N, h)
    psi = oracle.init_analytic(grid, 1, inputs.random_phase_field(*N, 6))
    a = oracle.observables(grid, Phys(g=0.0, omega=0.3), psi)
    b = oracle.observables(grid, Phys(g=10.0, omega=0.3), psi)
    q = 0.16 * np.sum(np.abs(psi) ** 4)
    assert abs((b["energy_c"] - a["energy_c"]) - 5.0 * q) < 1e-12
    assert abs((b["mu_c"] - a["mu_c"]) - 10.0 * q) < 1e-12


def test_rms_of_gaussian():
    N, h = 96, 0.125
    grid = Grid((N, N), (h, h))
    x, y = grid.coords(0)[None, :], grid.coords(1)[:, None]
    g1, n1 = 1.0, 1.7
    psi = np.exp(-(g1 * x ** 2 + n1 * y ** 2) / 2).astype(np.complex128)
    psi[0, :] = psi[:, 0] = 0
    ob = oracle.observables(grid, Phys(gamma=g1, nu=n1), psi)
    assert abs(ob["rms_x"] - np.sqrt(0.5 / g1)) < 1e-10
    assert abs(ob["rms_y"] - np.sqrt(0.5 / n1)) < 1e-10
    assert abs(ob["rms_r"] - np.sqrt(0.5 / g1 + 0.5 / n1)) < 1e-10
    # and the energy of this exact ground state is (gamma + nu)/2 to O(h^2)
    assert abs(ob["energy_c"] - (g1 + n1) / 2) < 5e-3


def test_rms_of_gaussian_3d():
    """The 3D anisotropic Gaussian exp(-(g x^2 + n y^2 + l z^2)/2) has
    <x^2> = 1/(2 g) and so on (rms of Sec. 2); its energy is (g + n + l)/2,
    reached at O(h^2) by the 3-point form and O(h^4) by the fourth-order one."""
    N, h = (40, 36, 44), (0.3, 0.3, 0.25)
    grid = Grid(N, h)
    x = grid.coords(0)[None, None, :]
    y = grid.coords(1)[None, :, None]
    z = grid.coords(2)[:, None, None]
    g1, n1, l1 = 1.0, 1.4, 0.8
    psi = np.exp(-(g1 * x ** 2 + n1 * y ** 2 + l1 * z ** 2) / 2).astype(np.complex128)
    psi[0, :, :] = psi[:, 0, :] = psi[:, :, 0] = 0
    ob = oracle.observables(grid, Phys(gamma=g1, nu=n1, lam=l1), psi)
    assert abs(ob["rms_x"] - np.sqrt(0.5 / g1)) < 1e-8
    assert abs(ob["rms_y"] - np.sqrt(0.5 / n1)) < 1e-8
    assert abs(ob["rms_z"] - np.sqrt(0.5 / l1)) < 1e-8
    assert abs(ob["rms_r"] - np.sqrt(0.5 / g1 + 0.5 / n1 + 0.5 / l1)) < 1e-8
    assert abs(ob["energy_c"] - (g1 + n1 + l1) / 2) < 1.5e-2  # O(h^2): -9.5e-3 here
    assert ob["max_density"] == 1.0  # the centre is a grid point
    # the fourth-order form converges at O(h^4): ratio ~16 per halving of h
    e1 = ob["energy4"] - (g1 + n1 + l1) / 2
    grid2 = Grid(tuple(2 * n for n in N), tuple(v / 2 for v in h))
    x = grid2.coords(0)[None, None, :]
    y = grid2.coords(1)[None, :, None]
    z = grid2.coords(2)[:, None, None]
    psi2 = np.exp(-(g1 * x ** 2 + n1 * y ** 2 + l1 * z ** 2) / 2).astype(np.complex128)
    psi2[0, :, :] = psi2[:, 0, :] = psi2[:, :, 0] = 0
    e2 = oracle.observables(grid2, Phys(gamma=g1, nu=n1, lam=l1), psi2)["energy4"] - (g1 + n1 + l1) / 2
    assert abs(e1) < 1e-3 and 12 < e1 / e2 < 20, (e1, e2)


@pytest.mark.parametrize("function,d", [(1, 1.0), (0, 1.0), (1, 1.3)])
def test_initial_state_normalisation(function, d):
    """Eq. fun: the Gaussian has unit norm, the one-vortex state norm d_xy^2."""
    N, h = 128, 0.125
    grid = Grid((N, N), (h, h))
    psi = oracle.init_analytic(grid, function, inputs.random_phase_field(N, N, 0),
                               d_xy=d, normalize=False)
    want = 1.0 if function == 0 else d * d
    assert abs(oracle.norm(grid, psi) - want) < 1e-10
    g3 = Grid((64, 64, 64), (0.2, 0.2, 0.1))
    psi3 = oracle.init_analytic(g3, function, inputs.random_phase_field(64, 64, 0),
                                d_xy=d, d_z=0.6, normalize=False)
    assert abs(oracle.norm(g3, psi3) - want) < 1e-9
    # the random phase leaves the density untouched
    plain = oracle.init_analytic(grid, function, None, d_xy=d, normalize=False)
    assert np.max(np.abs(np.abs(psi) - np.abs(plain))) < 1e-15


# ---------------------------------------------------------------- vortex count
def _vortex_state(grid, centres, charges):
    x, y = grid.coords(0)[None, :], grid.coords(1)[:, None]
    psi = np.exp(-(x ** 2 + y ** 2) / 8).astype(np.complex128)
    for (cx, cy), q in zip(centres, charges):
        z = (x - cx) + 1j * (y - cy)
        psi = psi * (z if q > 0 else np.conj(z))
    psi[0, :] = psi[-1, :] = psi[:, 0] = psi[:, -1] = 0
    return psi


@pytest.mark.parametrize("fp32", [False, True])
def test_vortex_count_on_constructed_states(fp32):
    grid = Grid((96, 96), (0.1, 0.1))
    cases = [([(0.03, 0.02)], [1], 1), ([(0.05, 0.05)], [-1], 1),
             ([(1.0, 0.3), (-1.0, 0.3), (0.05, -1.0)], [1, 1, 1], 3),
             ([(0.8, 0.0), (-0.8, 0.05)], [1, -1], 2), ([], [], 0)]
    for centres, charges, want in cases:
        psi = _vortex_state(grid, centres, charges)
        assert oracle.vortex_count(grid, psi, fp32) == want
    # 3D: the z = 0 plane is used
    g3 = Grid((32, 32, 8), (0.3, 0.3, 0.3))
    plane = _vortex_state(Grid((32, 32), (0.3, 0.3)),
                          [(0.55, 0.5), (-0.6, -0.4)], [1, 1])
    psi3 = np.repeat(plane[None, :, :], 9, axis=0)
    assert oracle.vortex_count(g3, psi3, fp32) == 2


# ------------------------------------------------- fourth-order energies
def _analytic_energies(n, h, function, omega):
    grid = Grid((n, n), (h, h))
    phys = Phys(gamma=1.0, nu=1.0, g=0.0, omega=omega, dt=1e-3)
    psi = oracle.init_analytic(grid, function, None)
    return oracle.observables(grid, phys, psi)


def test_fourth_order_energy_of_gaussian_is_exact_to_h4():
    """The isotropic harmonic ground state exp(-r^2/2)/sqrt(pi) has E = mu = 1
    (g = 0, Omega = 0).  With fourth-order differences the grid error is
    O(h^4): far below the O(h^2) error of the three-point forms, and it falls
    by ~16 when h halves (a wrong stencil coefficient breaks both)."""
    ob = _analytic_energies(128, 0.1, 0, 0.0)
    e4, e2 = abs(ob["energy4"] - 1.0), abs(ob["energy_c"] - 1.0)
    assert e4 < 3e-6 and e2 > 20 * e4, (e4, e2)
    assert abs(ob["mu4"] - ob["energy4"]) < 1e-13
    coarse = abs(_analytic_energies(64, 0.2, 0, 0.0)["energy4"] - 1.0)
    assert 12.0 < coarse / e4 < 20.0, coarse / e4


def test_fourth_order_energy_of_one_vortex_is_two_minus_omega():
    """(x + i y) exp(-r^2/2) is an L_z = +1 eigenstate with E = 2 - Omega
    (g = 0); the fourth-order evaluation includes the rotation term
    -Omega L_z through the fourth-order first derivatives."""
    omega = 0.5
    ob = _analytic_energies(128, 0.1, 1, omega)
    e4, e2 = abs(ob["energy4"] - (2 - omega)), abs(ob["energy_c"] - (2 - omega))
    assert e4 < 2e-5 and e2 > 20 * e4, (e4, e2)
    coarse = abs(_analytic_energies(64, 0.2, 1, omega)["energy4"] - (2 - omega))
    assert 12.0 < coarse / e4 < 20.0, coarse / e4


def test_fourth_order_forms_share_the_interaction_term():
    """mu - E is the interaction energy (g/2) sum |psi|^4 / sum |psi|^2 in
    both the three-point and the fourth-order complex forms."""
    n = (40, 36)
    grid = Grid(n, (0.3, 0.3))
    phys = Phys(gamma=1.0, nu=1.1, g=80.0, omega=0.6, dt=1e-3)
    psi = oracle.init_analytic(grid, 1, inputs.random_phase_field(n[0], n[1], 4))
    ob = oracle.observables(grid, phys, psi)
    assert abs((ob["mu4"] - ob["energy4"]) - (ob["mu_c"] - ob["energy_c"])) < 1e-12


@pytest.mark.parametrize("theta", [0.0, 0.4, 1.1, 2.6, np.pi / 2 - 0.01])
@pytest.mark.parametrize("shape", [(24, 20), (14, 12, 10)])
def test_real_part_forms_equal_complex_forms_on_a_phase_times_real_state(theta, shape):
    """For psi = e^{i theta} f with f real, the real-part forms of Eqs.
    e2dr/e3dr equal the complex forms of Eqs. e2d/e3d at any g and Omega:
    psi_R = cos(theta) f, so the interaction weight sum |psi|^2 psi_R^2 /
    sum psi_R^2 is sum f^4 / sum f^2 for both, and the rotation terms vanish
    in both because y D_x - x D_y is antisymmetric.  A wrong alpha (g/2 in E,
    g in mu), a wrong interaction weight or a wrong rotation sign in the
    real-part forms fails this.  theta close to pi/2 exercises the -i guard."""
    dim = len(shape)
    h = (0.4, 0.45, 0.5)[:dim]
    grid = Grid(shape, h)
    phys = Phys(gamma=1.0, nu=1.15, lam=1.3, g=37.0, omega=0.6, dt=2e-3)
    # f = |psi| of a rotating, interacting state (real and non-negative)
    psi = oracle.init_analytic(grid, 1, inputs.random_phase_field(shape[0], shape[1], 5))
    psi, _ = oracle.steps(grid, phys, psi, 60, True)
    f = np.abs(psi) * (1.0 + 0.2 * np.cos(np.arange(psi.size).reshape(psi.shape) * 0.37))
    state = np.exp(1j * theta) * f
    ob = oracle.observables(grid, phys, state)
    for a, b in (("energy", "energy_c"), ("mu", "mu_c")):
        assert abs(ob[a] - ob[b]) < 1e-12 * abs(ob[b]), (a, ob[a], ob[b])
    # the interaction contributes: the same state at g = 0 is far away
    ob0 = oracle.observables(grid, Phys(gamma=1.0, nu=1.15, lam=1.3, g=0.0, omega=0.6), state)
    assert abs(ob["energy"] - ob0["energy"]) > 0.1 and abs(ob["mu"] - ob0["mu"]) > 0.2


@pytest.mark.parametrize("shape", [(40, 36), (20, 18, 12)])
def test_initial_state_carries_the_random_phase_two_pi_r(shape):
    """Eq. fun multiplies the analytic state by exp(2 pi i R(x, y)): the phase
    of psi conj(psi without R) is 2 pi R_ij (mod 2 pi) at every interior point
    (i, j), the same on every z plane in 3D.  A phase of R instead of 2 pi R,
    or R indexed with x and y swapped, fails this."""
    dim = len(shape)
    grid = Grid(shape, (0.3, 0.25, 0.4)[:dim])
    R = inputs.random_phase_field(shape[0], shape[1], 11)
    psi = oracle.init_analytic(grid, 1, R, normalize=False)
    plain = oracle.init_analytic(grid, 1, None, normalize=False)
    prod = psi * np.conj(plain)
    ok = np.abs(plain) > 1e-12 * np.max(np.abs(plain))
    want = np.broadcast_to(R, prod.shape)  # R[j, i], x fastest; z planes share it
    d = np.angle(prod) - 2 * np.pi * want
    d = (d + np.pi) % (2 * np.pi) - np.pi
    assert ok.sum() > 0.5 * ok.size
    assert np.max(np.abs(d[ok])) < 1e-12
    # R is not symmetric, so a transposed index would not pass
    assert np.max(np.abs(R[:shape[0] + 1 - 4, :shape[0] + 1 - 4] -
                         R[:shape[0] + 1 - 4, :shape[0] + 1 - 4].T)) > 0.1
