"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances:
  FP64 path: max |psi_gpu - psi_oracle| <= 1e-10 after the same steps from
             the same seeded state; mu, E (real-part and complex) within
             1e-12 relative; identical vortex count.
  FP32 path (complex float bulk, FP64 reductions): relative L2 error of the
             density <= 1e-4, mu and E within 1e-5 relative, identical vortex
             count.
"""
import numpy as np
import pytest

import oracle
from oracle import Grid, Phys
from paper_1906_06327_gb300 import inputs
from paper_1906_06327_gb300.rotgp import (ROTGP_EINVAL, ROTGP_ENONFINITE, ROTGP_EUNSUPPORTED,
                                          RotgpError, Solver)

pytestmark = pytest.mark.gpu

OBS_REL = ("mu", "energy", "mu_c", "energy_c", "mu4", "energy4")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.init()


def _pair(n, h, phys: Phys, precision, function=1, seed=0, d_xy=1.0, d_z=1.0):
    """Oracle state and a solver holding the same state (init on the GPU)."""
    grid = Grid(n, h)
    R = inputs.random_phase_field(n[0], n[1], seed)
    psi0 = oracle.init_analytic(grid, function, R, d_xy, d_z)
    s = Solver(n, h, gamma=phys.gamma, nu=phys.nu, lam=phys.lam, g=phys.g, omega=phys.omega,
               dt=phys.dt, precision=precision)
    s.init_analytic(function, R, d_xy, d_z)
    return grid, psi0, s


def _rel_l2_density(a, b):
    da, db = np.abs(a) ** 2, np.abs(b) ** 2
    return np.linalg.norm(da - db) / np.linalg.norm(db)


def _check_fp64(s, grid, phys, psi_ref, tol_psi=1e-10, tol_rel=1e-12):
    psi = s.get_psi()
    assert np.max(np.abs(psi - psi_ref)) <= tol_psi
    ob = s.observables()
    ref = oracle.observables(grid, phys, psi_ref)
    for k in OBS_REL:
        assert abs(ob[k] - ref[k]) <= tol_rel * abs(ref[k]), (k, ob[k], ref[k])
    for k in ("norm", "rms_x", "rms_y", "rms_z", "rms_r"):
        assert abs(ob[k] - ref[k]) <= 1e-12 * max(1.0, abs(ref[k])), k
    assert ob["vortices"] == oracle.vortex_count(grid, psi_ref)
    return ob


def _check_fp32(s, grid, phys, psi_ref, tol_dens=1e-4, tol_rel=1e-5):
    psi = s.get_psi()
    assert _rel_l2_density(psi, psi_ref) <= tol_dens
    ob = s.observables()
    ref = oracle.observables(grid, phys, psi_ref)
    for k in OBS_REL:
        assert abs(ob[k] - ref[k]) <= tol_rel * abs(ref[k]), (k, ob[k], ref[k])
    assert abs(ob["norm"] - ref["norm"]) <= 1e-5
    assert ob["vortices"] == oracle.vortex_count(grid, psi_ref, fp32_decision=True)
    return ob


# ------------------------------------------------------------------ init / io
@pytest.mark.parametrize("n,h", [((128, 128), (0.1, 0.1)), ((37, 50), (0.3, 0.2)),
                                 ((20, 24, 18), (0.4, 0.35, 0.3))])
@pytest.mark.parametrize("function", [0, 1])
def test_init_analytic_matches_oracle(n, h, function):
    grid, psi0, s = _pair(n, h, Phys(), "fp64", function=function, seed=3, d_z=0.8)
    assert np.max(np.abs(s.get_psi() - psi0)) < 1e-14
    s32 = Solver(n, h, precision="fp32")
    s32.init_analytic(function, inputs.random_phase_field(n[0], n[1], 3), 1.0, 0.8)
    assert np.max(np.abs(s32.get_psi() - psi0)) < 2e-7 * np.max(np.abs(psi0)) * 4


def test_set_get_roundtrip_and_edges():
    n, h = (33, 17), (0.2, 0.3)
    rng = np.random.default_rng(0)
    shape = (n[1] + 1, n[0] + 1)
    psi = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    s = Solver(n, h, precision="fp64")
    s.set_psi(psi)
    out = s.get_psi()
    inner = (slice(1, -1), slice(1, -1))
    assert np.array_equal(out[inner], psi[inner])
    assert not out[0, :].any() and not out[-1, :].any()
    assert not out[:, 0].any() and not out[:, -1].any()
    s.set_psi(psi.astype(np.complex64))
    out32 = s.get_psi(fp64=False)
    assert out32.dtype == np.complex64
    assert np.array_equal(out32[inner], psi.astype(np.complex64)[inner])


def test_device_buffers_through_torch():
    import torch
    n, h = (40, 30), (0.25, 0.25)
    grid, psi0, s = _pair(n, h, Phys(g=10.0, omega=0.3, dt=1e-3), "fp64")
    t = torch.zeros(s.shape, dtype=torch.complex128, device="cuda")
    s.get_psi(t)
    assert np.max(np.abs(t.cpu().numpy() - psi0)) < 1e-14
    t32 = torch.zeros(s.shape, dtype=torch.complex64, device="cuda")
    s.get_psi(t32)
    s2 = Solver(n, h, precision="fp64")
    s2.set_psi(t)
    assert np.max(np.abs(s2.get_psi() - psi0)) < 1e-14


# ------------------------------------------------------------------ one step
@pytest.mark.parametrize("n,h", [((4, 4), (0.9, 0.8)), ((5, 7), (0.8, 0.6)),
                                 ((33, 65), (0.25, 0.12)), ((100, 31), (0.1, 0.3)),
                                 ((6, 5, 4), (0.9, 0.8, 0.7)), ((35, 9, 70), (0.2, 0.6, 0.1))])
@pytest.mark.parametrize("imag", [True, False])
def test_single_step_fp64_small_and_ragged(n, h, imag):
    phys = Phys(gamma=1.0, nu=1.3, lam=0.9, g=20.0, omega=0.6, dt=0.02)
    grid, psi0, s = _pair(n, h, phys, "fp64", seed=11)
    ref, _ = oracle.steps(grid, phys, psi0, 1, imag)
    (s.step_imag if imag else s.step_real)(1)
    assert np.max(np.abs(s.get_psi() - ref)) <= 1e-13


@pytest.mark.parametrize("n,h", [((5, 7), (0.8, 0.6)), ((100, 31), (0.1, 0.3)),
                                 ((35, 9, 70), (0.2, 0.6, 0.1))])
@pytest.mark.parametrize("imag", [True, False])
def test_single_step_fp32_small_and_ragged(n, h, imag):
    phys = Phys(gamma=1.0, nu=1.3, lam=0.9, g=20.0, omega=0.6, dt=0.02)
    grid, psi0, s = _pair(n, h, phys, "fp32", seed=11)
    ref, _ = oracle.steps(grid, phys, psi0, 1, imag)
    (s.step_imag if imag else s.step_real)(1)
    psi = s.get_psi()
    assert np.max(np.abs(psi - ref)) <= 2e-6 * np.max(np.abs(ref))


# ------------------------------------------------------------------ the 128^2 FP64 run
def test_imaginary_time_2d_128_fp64_1000_steps():
    """2D, 128^2, dx = 0.1, gamma = nu = 1, g = 100, Omega = 0.5, dt = 1e-3,
    1000 imaginary-time steps from the seed-0 one-vortex random-phase state."""
    w = inputs.WL_2D_128_FP64
    phys = Phys(gamma=w.gamma, nu=w.nu, lam=w.lam, g=w.g, omega=w.omega, dt=w.dt)
    grid, psi0, s = _pair(w.n, w.h, phys, "fp64", seed=w.seed)
    ref, _ = oracle.steps(grid, phys, psi0, w.imag_steps, True)
    s.step_imag(w.imag_steps)
    _check_fp64(s, grid, phys, ref)


def test_real_time_2d_fp64_conserves_and_matches():
    n, h = (96, 80), (0.12, 0.15)
    phys = Phys(gamma=1.0, nu=1.1, g=60.0, omega=0.7, dt=1e-3)
    grid, psi0, s = _pair(n, h, phys, "fp64", seed=5)
    s.step_imag(200)
    psi_start = s.get_psi()
    ref, nrm = oracle.steps(grid, phys, psi_start, 400, False)
    s.step_real(400)
    ob = _check_fp64(s, grid, phys, ref)
    assert abs(ob["norm"] - 1.0) < 1e-12


def test_imaginary_time_3d_fp64_ragged():
    n, h = (40, 36, 22), (0.3, 0.3, 0.25)
    phys = Phys(gamma=1.0, nu=1.05, lam=1.5, g=150.0, omega=0.6, dt=2e-3)
    grid, psi0, s = _pair(n, h, phys, "fp64", seed=7, d_z=0.8)
    ref, _ = oracle.steps(grid, phys, psi0, 150, True)
    s.step_imag(150)
    _check_fp64(s, grid, phys, ref)


# ------------------------------------------------------------------ FP32 runs
def test_imaginary_time_2d_fp32():
    n, h = (160, 96), (0.1, 0.12)
    phys = Phys(gamma=1.0, nu=1.05, g=300.0, omega=0.8, dt=5e-4)
    grid, psi0, s = _pair(n, h, phys, "fp32", seed=2)
    ref, _ = oracle.steps(grid, phys, psi0, 600, True)
    s.step_imag(600)
    _check_fp32(s, grid, phys, ref)


def test_real_time_3d_fp32():
    n, h = (48, 40, 36), (0.25, 0.25, 0.2)
    phys = Phys(gamma=1.0, nu=1.0, lam=0.8, g=200.0, omega=0.7, dt=1e-3)
    grid, psi0, s = _pair(n, h, phys, "fp32", seed=4, d_z=1.0)
    s.step_imag(50)
    start = s.get_psi()
    ref, _ = oracle.steps(grid, phys, start, 100, False)
    s.step_real(100)
    ob = _check_fp32(s, grid, phys, ref)
    assert abs(ob["norm"] - 1.0) < 1e-5


# ------------------------------------------------------------------ observables
@pytest.mark.parametrize("n,h", [((64, 48), (0.2, 0.25)), ((30, 26, 20), (0.35, 0.4, 0.3))])
def test_observables_on_identical_state(n, h):
    phys = Phys(gamma=1.0, nu=1.2, lam=1.3, g=80.0, omega=0.55, dt=1e-3)
    grid = Grid(n, h)
    psi = oracle.init_analytic(grid, 1, inputs.random_phase_field(n[0], n[1], 9))
    psi, _ = oracle.steps(grid, phys, psi, 300, True)
    ref = oracle.observables(grid, phys, psi)
    for prec, tol in (("fp64", 1e-12), ("fp32", 2e-6)):
        s = Solver(n, h, gamma=1.0, nu=1.2, lam=1.3, g=80.0, omega=0.55, dt=1e-3,
                   precision=prec)
        s.set_psi(psi)
        ob = s.observables()
        for k in OBS_REL + ("rms_x", "rms_y", "rms_r", "max_density"):
            assert abs(ob[k] - ref[k]) <= tol * abs(ref[k]), (prec, k)
        assert ob["vortices"] == oracle.vortex_count(grid, psi, fp32_decision=prec == "fp32")
    # a state with global phase i exercises the real-part guard
    s = Solver(n, h, gamma=1.0, nu=1.2, lam=1.3, g=80.0, omega=0.55, dt=1e-3, precision="fp64")
    real_state = np.abs(psi).astype(np.complex128)
    s.set_psi(1j * real_state)
    ref_i = oracle.observables(grid, phys, 1j * real_state)
    assert abs(s.observables()["energy"] - ref_i["energy"]) <= 1e-12 * abs(ref_i["energy"])


def test_vortex_count_on_lattice_state():
    """A converged multi-vortex state: GPU count equals the oracle's."""
    n, h = (128, 128), (0.1, 0.1)
    phys = Phys(g=200.0, omega=0.85, dt=2e-3)
    grid, psi0, s = _pair(n, h, phys, "fp64", seed=1)
    s.step_imag(3000)
    psi = s.get_psi()
    ob = s.observables()
    want = oracle.vortex_count(grid, psi)
    assert ob["vortices"] == want
    assert want >= 1


# ------------------------------------------------------------------ errors
def test_error_paths():
    with pytest.raises(RotgpError) as e:
        Solver((8, 8), (0.1, -0.1))
    assert e.value.code == ROTGP_EINVAL
    with pytest.raises(RotgpError) as e:
        Solver((256, 256), (0.001, 0.001), dt=1.0)  # Delta/h^2 = 1e6
    assert e.value.code == ROTGP_EUNSUPPORTED
    s = Solver((16, 16), (0.3, 0.3), g=10.0, precision="fp32")
    bad = np.zeros(s.shape, dtype=np.complex128)
    bad[5, 5] = np.nan
    s.set_psi(bad)
    s.step_imag(1)
    with pytest.raises(RotgpError) as e:
        s.observables()
    assert e.value.code == ROTGP_ENONFINITE
    # a fresh state clears the flag
    s.init_analytic(1, None)
    s.step_imag(2)
    assert abs(s.observables()["norm"] - 1.0) < 1e-6
    with pytest.raises(RotgpError):
        s.step_imag(-1)


# ------------------------------------------------------------------ full size
@pytest.mark.slow
def test_3d_256x256x128_fp32_two_steps_full_grid():
    """The 3D FP32 workload at full size (256 x 256 x 128, the launch
    configuration the benchmark times): two imaginary-time steps from the
    seeded start, every point compared with the oracle."""
    w = inputs.WL_3D_256_FP32
    phys = Phys(gamma=w.gamma, nu=w.nu, lam=w.lam, g=w.g, omega=w.omega, dt=w.dt)
    grid, psi0, s = _pair(w.n, w.h, phys, "fp32", seed=w.seed)
    ref, _ = oracle.steps(grid, phys, psi0, 2, True)
    s.step_imag(2)
    psi = s.get_psi()
    assert _rel_l2_density(psi, ref) <= 1e-5
    assert np.max(np.abs(psi - ref)) <= 1e-6 * np.max(np.abs(ref)) * 8
    ob = s.observables()
    refo = oracle.observables(grid, phys, ref)
    for k in OBS_REL:
        assert abs(ob[k] - refo[k]) <= 1e-5 * abs(refo[k]), k


# ------------------------------------------------------------------ solver forms
@pytest.mark.parametrize("n,h", [((100, 64), (0.12, 0.15)), ((132, 36), (0.1, 0.3)),
                                 ((130, 70), (0.1, 0.12)), ((44, 36, 40), (0.3, 0.3, 0.25)),
                                 ((70, 50, 46), (0.2, 0.22, 0.25))])
@pytest.mark.parametrize("imag", [True, False])
def test_stencil_forms_match_thomas_fp32(n, h, imag):
    """The fused H1 + x + y tile pass, the separate stencil sweeps and the
    Thomas solve are the same split step: same state after 20 steps up to
    float rounding, on grids whose tiles do not divide them."""
    phys = dict(gamma=1.0, nu=1.1, lam=1.3, g=120.0, omega=0.7, dt=1e-3)
    R = inputs.random_phase_field(n[0], n[1], 8)
    forms = {}
    fused = Solver(n, h, precision="fp32", **phys)
    fused.set_solver(0, "fused")
    for axis in range(2, len(n)):
        fused.set_solver(axis, "stencil")
    info = fused.info()
    assert info["fused_xy"] == 1 and all(t > 0 for t in info["stencil_taps"]), info
    forms["fused"] = fused
    if n[0] % 4 == 0:
        sep = Solver(n, h, precision="fp32", **phys)
        for axis in range(len(n)):
            sep.set_solver(axis, "stencil")
        assert sep.info()["fused_xy"] == 0
        forms["stencil"] = sep
    if len(n) == 3 or n[1] >= 48:
        seg = Solver(n, h, precision="fp32", **phys)
        for axis in range(1, len(n)):
            seg.set_solver(axis, "stencil")
            seg.tune(axis, 2, 8, 3, 1, 3)  # three segments per line (ragged)
            assert seg.info()["segments"][axis] == 3
        forms["stencil_segments"] = seg
    th = Solver(n, h, precision="fp32", **phys)  # the default form
    assert all(t == 0 for t in th.info()["stencil_taps"]) and th.info()["fused_xy"] == 0
    forms["thomas"] = th
    psi = {}
    for k, s in forms.items():
        s.init_analytic(1, R, 1.0, 1.0)
        (s.step_imag if imag else s.step_real)(20)
        psi[k] = s.get_psi()
    grid = Grid(n, h)
    ref, _ = oracle.steps(grid, Phys(gamma=1.0, nu=1.1, lam=1.3, g=120.0, omega=0.7, dt=1e-3),
                          oracle.init_analytic(grid, 1, R), 20, imag)
    # float rounding of different evaluation orders over 20 steps of a rough
    # random-phase state (the stencil's truncated tail is below 2e-10)
    scale = np.max(np.abs(ref))
    for k, p in psi.items():
        assert np.max(np.abs(p - psi["thomas"])) <= 5e-6 * scale, k
        assert np.max(np.abs(p - ref)) <= 5e-6 * scale, k
    # the zero edges stay exactly zero
    for p in psi.values():
        for ax in range(len(n)):
            assert np.all(np.take(p, [0, n[ax]], axis=len(n) - 1 - ax) == 0)


def test_fused_pass_selection():
    """Selecting a per-axis solver turns the fused pass off; FUSED turns it
    back on; FUSED is refused on z."""
    s = Solver((64, 48, 32), (0.2, 0.2, 0.25), precision="fp32", gamma=1.0, nu=1.0, lam=1.0,
               g=50.0, omega=0.5, dt=1e-3)
    assert s.info()["fused_xy"] == 0
    s.set_solver(0, "fused")
    assert s.info()["fused_xy"] == 1
    s.set_solver(1, "thomas")
    assert s.info()["fused_xy"] == 0 and s.info()["stencil_taps"][1] == 0
    s.set_solver(0, "fused")
    assert s.info()["fused_xy"] == 1 and s.info()["stencil_taps"][1] > 0
    with pytest.raises(RotgpError):
        s.set_solver(2, "fused")
    d = Solver((64, 48), (0.2, 0.2), precision="fp64", gamma=1.0, nu=1.0, g=50.0, omega=0.5,
               dt=1e-3)
    assert d.info()["fused_xy"] == 0
    with pytest.raises(RotgpError):
        d.set_solver(0, "fused")


@pytest.mark.parametrize("n,h", [((96, 64), (0.12, 0.15)), ((40, 36, 32), (0.3, 0.3, 0.25))])
def test_autotune_restores_state_and_keeps_parity(n, h):
    """The autotuner times the forms on a copy of the state: the state, the
    step counter and the results of later steps are those of an untuned
    context up to float rounding."""
    phys = dict(gamma=1.0, nu=1.1, lam=1.3, g=120.0, omega=0.7, dt=1e-3)
    R = inputs.random_phase_field(n[0], n[1], 3)
    a = Solver(n, h, precision="fp32", **phys)
    b = Solver(n, h, precision="fp32", **phys)
    for s in (a, b):
        s.init_analytic(1, R, 1.0, 1.0)
        s.step_imag(3)
    before = a.get_psi()
    choice = a.autotune(steps=2)
    assert set(choice["forms"]) <= {"thomas", "stencil", "fused"}
    assert np.array_equal(a.get_psi(), before)
    assert a.observables()["step"] == 3
    for s in (a, b):
        s.step_imag(10)
    pa, pb = a.get_psi(), b.get_psi()
    assert np.max(np.abs(pa - pb)) <= 5e-6 * np.max(np.abs(pb))


def test_bounded_wait_gives_up_and_context_stays_usable():
    """A device wait that can never be satisfied gives up by itself (about
    2 s of device time) and the kernel returns normally; the context then
    still steps correctly."""
    from paper_1906_06327_gb300.rotgp import check_bounded_wait
    sec = check_bounded_wait()
    assert 0.5 < sec < 10.0, sec
    n, h = (40, 36), (0.3, 0.3)
    s = Solver(n, h, precision="fp32", gamma=1.0, nu=1.0, g=20.0, omega=0.3, dt=1e-3)
    s.init_analytic(1, inputs.random_phase_field(n[0], n[1], 0), 1.0, 1.0)
    s.step_imag(5)
    assert abs(s.observables()["norm"] - 1.0) < 1e-5


@pytest.mark.parametrize("shape", [(1, 8, 3, 2), (1, 16, 4, 3), (1, 8, 6, 2), (2, 8, 3, 2),
                                   (2, 16, 4, 1)])
@pytest.mark.parametrize("n,h", [((100, 64), (0.12, 0.15)), ((46, 36, 30), (0.3, 0.3, 0.25))])
@pytest.mark.parametrize("imag", [True, False])
def test_thomas_x_launch_shapes_fp32(shape, n, h, imag):
    """Every launch shape of the Thomas x sweep (one or two rows per lane,
    chunk, ring, segments) gives the oracle's state after 20 steps up to
    float rounding."""
    V, C, R, sg = shape
    phys = dict(gamma=1.0, nu=1.1, lam=1.3, g=120.0, omega=0.7, dt=1e-3)
    R_ = inputs.random_phase_field(n[0], n[1], 5)
    s = Solver(n, h, precision="fp32", **phys)
    s.tune(0, V, C, R, 1, sg)
    info = s.info()
    assert (info["lines_per_lane"][0], info["chunk"][0], info["ring"][0]) == (V, C, R)
    s.init_analytic(1, R_, 1.0, 1.0)
    (s.step_imag if imag else s.step_real)(20)
    grid = Grid(n, h)
    ref, _ = oracle.steps(grid, Phys(**phys), oracle.init_analytic(grid, 1, R_), 20, imag)
    assert np.max(np.abs(s.get_psi() - ref)) <= 5e-6 * np.max(np.abs(ref))


def test_tma_sweeps_with_several_units_per_warp():
    """Launch shapes whose 32-line units (4096 per sweep) outnumber the
    resident persistent warps, so that every warp solves units in turn with
    its ring's barrier phases and pending stores carried from one unit to
    the next, match the oracle after two imaginary-time steps."""
    n, h = (128, 128, 64), (0.12, 0.12, 0.14)
    phys = dict(gamma=1.0, nu=1.1, lam=1.3, g=120.0, omega=0.7, dt=1e-3)
    s = Solver(n, h, precision="fp32", **phys)
    s.tune(0, 1, 8, 5, 1, 16)
    s.tune(1, 1, 8, 5, 1, 16)
    s.tune(2, 1, 8, 5, 1, 8)
    info = s.info()
    assert info["segments"] == [16, 16, 8] and info["lines_per_lane"] == [1, 1, 1]
    R_ = inputs.random_phase_field(n[0], n[1], 7)
    s.init_analytic(1, R_, 1.0, 1.0)
    s.step_imag(2)
    grid = Grid(n, h)
    ref, _ = oracle.steps(grid, Phys(**phys), oracle.init_analytic(grid, 1, R_), 2, True)
    assert np.max(np.abs(s.get_psi() - ref)) <= 5e-6 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", [(1, 8, 3, 2), (1, 16, 4, 3), (2, 8, 3, 2), (1, 8, 4, 1),
                                   (1, 8, 5, 3), (1, 8, 6, 1)])
@pytest.mark.parametrize("n,h", [((100, 66), (0.12, 0.15)), ((46, 36, 30), (0.3, 0.3, 0.25))])
@pytest.mark.parametrize("imag", [True, False])
def test_thomas_yz_launch_shapes_fp32(shape, n, h, imag):
    """Every launch shape of the Thomas y and z sweeps (one or two lines per
    lane, chunk, ring, segments; the last sweep also reduces the norm) gives
    the oracle's state after 20 steps up to float rounding."""
    V, C, R, sg = shape
    phys = dict(gamma=1.0, nu=1.1, lam=1.3, g=120.0, omega=0.7, dt=1e-3)
    R_ = inputs.random_phase_field(n[0], n[1], 6)
    s = Solver(n, h, precision="fp32", **phys)
    for ax in range(1, len(n)):
        s.tune(ax, V, C, R, 1, sg)
    info = s.info()
    for ax in range(1, len(n)):
        assert (info["lines_per_lane"][ax], info["chunk"][ax], info["ring"][ax]) == (V, C, R)
    s.init_analytic(1, R_, 1.0, 1.0)
    (s.step_imag if imag else s.step_real)(20)
    grid = Grid(n, h)
    ref, _ = oracle.steps(grid, Phys(**phys), oracle.init_analytic(grid, 1, R_), 20, imag)
    assert np.max(np.abs(s.get_psi() - ref)) <= 5e-6 * np.max(np.abs(ref))
    ob, refo = s.observables(), oracle.observables(grid, Phys(**phys), ref)
    assert abs(ob["norm"] - refo["norm"]) <= 1e-5


# ------------------------------------------------------------------ Omega(t)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("imag", [False, True])
def test_omega_schedule_matches_oracle(precision, imag):
    """rotgp_step_schedule: step k at Omega_k (a linear ramp 0.75 -> 0.6 held
    fixed within each step, as the real-time runs of Sec. 3 change Omega)
    equals the oracle stepping one step at a time with the same Omega_k."""
    n, h = (64, 48), (0.25, 0.3)
    phys = Phys(gamma=1.0, nu=1.1, g=30.0, omega=0.75, dt=2e-3)
    grid, psi, s = _pair(n, h, phys, precision, seed=6)
    om = 0.75 - 0.15 * np.arange(40) / 40
    for w in om:
        psi, _ = oracle.steps(grid, Phys(gamma=1.0, nu=1.1, g=30.0, omega=float(w), dt=2e-3), psi,
                              1, imag)
    s.step_schedule(om, imag=imag)
    end = Phys(gamma=1.0, nu=1.1, g=30.0, omega=float(om[-1]), dt=2e-3)
    (_check_fp64 if precision == "fp64" else _check_fp32)(s, grid, end, psi)
    # the context keeps the last Omega: one more plain step matches too
    psi, _ = oracle.steps(grid, end, psi, 1, imag)
    (s.step_imag if imag else s.step_real)(1)
    (_check_fp64 if precision == "fp64" else _check_fp32)(s, grid, end, psi)


def test_omega_schedule_beyond_the_plan_is_refused():
    s = Solver((64, 64), (0.05, 0.05), g=10.0, omega=0.1, dt=5e-3, precision="fp32")
    with pytest.raises(RotgpError) as e:
        s.step_schedule(np.array([0.1, 5.0, 0.1]))
    assert e.value.code == ROTGP_EUNSUPPORTED


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("n,h", [((30, 26, 20), (0.35, 0.4, 0.3)), ((40, 36), (0.3, 0.3))])
def test_column_density_matches_oracle(precision, n, h):
    """rotgp_column_density: h_z sum_k |psi|^2 (the reduced density of the
    3D lattices of Sec. 3), or the density in 2D, against the oracle state."""
    phys = Phys(gamma=1.0, nu=1.1, lam=1.4, g=30.0, omega=0.5, dt=2e-3)
    grid, psi, s = _pair(n, h, phys, precision, seed=8)
    psi, _ = oracle.steps(grid, phys, psi, 10, True)
    s.step_imag(10)
    col = s.column_density()
    dens = np.abs(psi) ** 2
    want = dens.sum(axis=0) * h[2] if len(n) == 3 else dens
    tol = 1e-12 if precision == "fp64" else 2e-6
    assert np.max(np.abs(col - want)) <= tol * np.max(want)
    assert abs(col.sum() * h[0] * h[1] - 1.0) < (1e-12 if precision == "fp64" else 1e-5)
