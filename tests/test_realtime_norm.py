"""Real-time norm conservation of the complex-float CN map, per solver form
(Eqs. eqD.9-eqD.11 and eq1 of the paper: both substeps are unitary in exact
arithmetic).  Each form runs 100,000 real-time steps of Delta = 1e-4 from a
smoothed seeded state and must keep the norm within 1e-9 per step; the
rounding effects the kernels avoid (a near-unit coefficient rounded to
float, the H1 rotation rounded on its own, large terms rounded once per
small term) each drifted by 1e-9 to 2e-8 per step on such states."""
import numpy as np
import pytest

from paper_1906_06327_gb300.rotgp import Batch, Solver

pytestmark = pytest.mark.gpu

PER_STEP = 1e-9
STEPS = 100_000


def _smoothed(s, lam):
    s.init_analytic(1, seed=7, d_z=lam ** -0.5)
    s.step_imag(2000)


@pytest.mark.parametrize("forms", [None, "hybrid"])
def test_2d_norm_per_step(forms):
    kw = dict(gamma=1.0, nu=1.0, g=100.0, omega=0.8)
    s = Solver((128, 128), (0.1, 0.1), dt=1e-3, **kw)
    _smoothed(s, 1.0)
    s.set_phys(dt=1e-4, **kw)
    if forms:
        s.set_solver(0, forms)
        s.set_solver(1, forms)
    n0 = s.observables()["norm"]
    s.step_real(STEPS)
    n1 = s.observables()["norm"]
    assert abs(n1 - n0) < PER_STEP * STEPS, (forms, n0, n1)


@pytest.mark.parametrize("forms", [None, "hybrid"])
def test_3d_norm_per_step(forms):
    kw = dict(gamma=1.0, nu=1.0, lam=4.0, g=50.0, omega=0.6)
    s = Solver((64, 64, 32), (0.2, 0.2, 0.1), dt=1e-3, **kw)
    _smoothed(s, 4.0)
    s.set_phys(dt=1e-4, **kw)
    if forms:
        for a in range(3):
            s.set_solver(a, forms)
    n0 = s.observables()["norm"]
    s.step_real(STEPS // 4)
    n1 = s.observables()["norm"]
    assert abs(n1 - n0) < PER_STEP * STEPS / 4, (forms, n0, n1)


def test_persistent_batch_norm_per_step():
    sp = dict(n=(128, 128), h=(0.1, 0.1), gamma=1.0, nu=1.0, g=100.0, omega=0.8, dt=1e-3)
    b = Batch([sp, dict(sp, n=(96, 96), h=(0.13, 0.13), omega=0.6)])
    for inst in b.instances:
        inst.init_analytic(1, seed=7)
    b.step_imag(2000, mode="persistent")
    for inst, p in zip(b.instances, (sp, dict(sp, omega=0.6))):
        inst.set_phys(gamma=1.0, nu=1.0, g=100.0, omega=p["omega"], dt=1e-4)
    n0 = np.array([o["norm"] for o in b.observables()])
    b.step_real(STEPS, mode="persistent")
    n1 = np.array([o["norm"] for o in b.observables()])
    b.close()
    assert np.all(np.abs(n1 - n0) < PER_STEP * STEPS), (n0, n1)
