"""Batched instances (rotgp_batch_*): the same steps as single contexts, bit
for bit, with and without CUDA graphs; convergence bookkeeping; argument
errors (CPU)."""
import numpy as np
import pytest

from paper_1906_06327_gb300 import inputs
from paper_1906_06327_gb300.rotgp import Batch, RotgpError, Solver, load

SPECS = [
    dict(n=(64, 48), h=(0.2, 0.25), gamma=1.0, nu=1.05, g=80.0, omega=0.6, dt=1e-3),
    dict(n=(100, 80), h=(0.15, 0.16), gamma=1.0, nu=1.1, g=200.0, omega=0.8, dt=1e-3),
    dict(n=(36, 32, 28), h=(0.3, 0.3, 0.35), gamma=1.0, nu=1.0, lam=1.4, g=60.0, omega=0.5,
         dt=1e-3),
]
# solver forms per instance: Thomas; fused x-y pass; Thomas x/y + stencil z
FORMS = [{}, {0: "fused"}, {2: "stencil"}]


def _forms(s, forms):
    for ax, f in forms.items():
        s.set_solver(ax, f)


def test_batch_rejects_bad_arguments():
    lib = load()
    import ctypes
    h = ctypes.c_void_p()
    assert lib.rotgp_batch_create(0, None, None, 1, None, ctypes.byref(h)) != 0
    assert lib.rotgp_batch_step(None, 1, 1, 1) != 0
    assert lib.rotgp_batch_count(None) == 0


@pytest.mark.gpu
@pytest.mark.parametrize("graph", [True, False])
def test_batch_matches_single_contexts_bitwise(graph):
    b = Batch(SPECS)
    singles = []
    for i, sp in enumerate(SPECS):
        kw = {k: v for k, v in sp.items() if k not in ("n", "h")}
        s = Solver(sp["n"], sp["h"], **kw)
        R = inputs.random_phase_field(sp["n"][0], sp["n"][1], 10 + i)
        for x in (s, b.instances[i]):
            _forms(x, FORMS[i])
            x.init_analytic(1, R, 1.0, 1.0)
        singles.append(s)
    # 7 + 7 + 6 steps: odd blocks exercise both buffer parities of a graph
    b.step_imag(7, graph=graph)
    b.step_imag(7, graph=graph)
    b.step_imag(6, graph=graph)
    b.step_real(3, graph=graph)
    for s in singles:
        s.step_imag(20)
        s.step_real(3)
    obs = b.observables()
    for i, s in enumerate(singles):
        assert np.array_equal(b.instances[i].get_psi(), s.get_psi()), i
        assert obs[i]["step"] == 23
        assert obs[i]["mu"] == s.observables()["mu"]
    b.close()


@pytest.mark.gpu
def test_batch_converge_bookkeeping():
    specs = [dict(n=(48, 48), h=(0.25, 0.25), gamma=1.0, nu=1.0, g=10.0, omega=0.2, dt=2e-3),
             dict(n=(64, 40), h=(0.2, 0.3), gamma=1.0, nu=1.1, g=40.0, omega=0.4, dt=2e-3)]
    b = Batch(specs)
    for i, sp in enumerate(specs):
        b.instances[i].init_analytic(0, None, 1.0, 1.0)  # Gaussian start, no vortices
    steps, conv = b.converge(1e-4, 100, 20000)
    assert all(conv), (steps, conv)
    assert all(0 < s <= 20000 and s % 100 == 0 for s in steps)
    obs = b.observables()
    for i, o in enumerate(obs):
        assert o["step"] == steps[i]
        # a converged instance gained nothing more: one more check window moves mu little
    b.step_imag(100)
    obs2 = b.observables()
    for o, o2 in zip(obs, obs2):
        assert abs(o2["mu"] - o["mu"]) <= 1e-3 * abs(o["mu"])
    b.close()


# ------------------------------------------------------------------ persistent
SPECS2D = [
    dict(n=(64, 48), h=(0.2, 0.25), gamma=1.0, nu=1.05, g=80.0, omega=0.6, dt=1e-3),
    dict(n=(100, 80), h=(0.15, 0.16), gamma=1.0, nu=1.1, g=200.0, omega=0.8, dt=1e-3),
    dict(n=(37, 50), h=(0.3, 0.22), gamma=1.0, nu=1.0, g=40.0, omega=0.4, dt=2e-3),
    dict(n=(256, 192), h=(0.06, 0.08), gamma=1.0, nu=1.02, g=500.0, omega=0.9, dt=5e-4),
]


def _hybrid_whole_lines(s):
    """The exact line solve on both axes, one CTA per line (the persistent
    batch step's form)."""
    for ax in (0, 1):
        s.set_solver(ax, "hybrid")
        s.tune(ax, 1, 8, 3, 1, 1)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_persistent_batch_matches_single_contexts_bitwise(precision):
    """One cooperative launch per block of steps over all instances equals,
    bit for bit, each instance stepped alone with the same line solve."""
    b = Batch(SPECS2D, precision=precision)
    singles = []
    for i, sp in enumerate(SPECS2D):
        kw = {k: v for k, v in sp.items() if k not in ("n", "h")}
        s = Solver(sp["n"], sp["h"], precision=precision, **kw)
        _hybrid_whole_lines(s)
        s.init_analytic(1, seed=20 + i)
        b.instances[i].init_analytic(1, seed=20 + i)
        singles.append(s)
    b.step_imag(7, mode="persistent")
    b.step_imag(13, mode="persistent")
    b.step_real(3, mode="persistent")
    for s in singles:
        s.step_imag(7)
        s.step_imag(13)
        s.step_real(3)
    obs = b.observables()
    for i, s in enumerate(singles):
        assert np.array_equal(b.instances[i].get_psi(), s.get_psi()), i
        o = s.observables()
        assert obs[i]["step"] == 23 and obs[i]["mu"] == o["mu"] and obs[i]["norm"] == o["norm"]
    b.close()


@pytest.mark.gpu
def test_persistent_batch_fp64_matches_oracle():
    import oracle
    from oracle import Grid, Phys
    b = Batch(SPECS2D[:3], precision="fp64")
    refs = []
    for i, sp in enumerate(SPECS2D[:3]):
        grid = Grid(sp["n"], sp["h"])
        phys = Phys(gamma=sp["gamma"], nu=sp["nu"], g=sp["g"], omega=sp["omega"], dt=sp["dt"])
        R = inputs.random_phase_field(sp["n"][0], sp["n"][1], 30 + i)
        b.instances[i].init_analytic(1, R)
        ref, _ = oracle.steps(grid, phys, oracle.init_analytic(grid, 1, R), 20, True)
        ref, _ = oracle.steps(grid, phys, ref, 5, False)
        refs.append((grid, phys, ref))
    b.step_imag(20, mode="persistent")
    b.step_real(5, mode="persistent")
    obs = b.observables()
    for i, (grid, phys, ref) in enumerate(refs):
        assert np.max(np.abs(b.instances[i].get_psi() - ref)) < 1e-10, i
        r = oracle.observables(grid, phys, ref)
        assert abs(obs[i]["mu"] - r["mu"]) < 1e-12 * abs(r["mu"]), i
    b.close()


@pytest.mark.gpu
def test_persistent_batch_converges_and_refuses_3d():
    specs = [dict(n=(48, 48), h=(0.25, 0.25), gamma=1.0, nu=1.0, g=10.0, omega=0.2, dt=2e-3),
             dict(n=(64, 40), h=(0.2, 0.3), gamma=1.0, nu=1.1, g=40.0, omega=0.4, dt=2e-3)]
    b = Batch(specs)
    for i in range(2):
        b.instances[i].init_analytic(0, None, 1.0, 1.0)
    steps, conv = b.converge(1e-4, 100, 20000, mode="persistent")
    assert all(conv), (steps, conv)
    obs = b.observables()
    for i, o in enumerate(obs):
        assert o["step"] == steps[i]
    b.close()
    b3 = Batch([dict(n=(16, 16, 16), h=(0.3, 0.3, 0.3), g=10.0, dt=1e-3)])
    with pytest.raises(RotgpError) as e:
        b3.step_imag(1, mode="persistent")
    assert e.value.code == -5  # ROTGP_EUNSUPPORTED
    b3.close()
