"""The real-time norm bounds used by the long-run physics tests, derived on
the CPU from the CN amplification factor (Eqs. eqD.9-eqD.11 and eq5 of the
paper).

In the interior of a line, where the Thomas multipliers have reached their
fixed point, the folded forward recurrence d_p = (1 + a0) psi_p + am
psi_{p-1} + ap psi_{p+1} + al d_{p-1} and the backward one x_p = d_p + be
x_{p+1} map the Fourier mode e^{ikp} to G(k) e^{ikp} with

    G(k) = ((1 + a0) + am e^{-ik} + ap e^{ik}) / ((1 - al e^{-ik}) (1 - be e^{ik})),

and |G(k)| = 1 for every k in exact arithmetic (the CN map of a Hermitian
operator is unitary).  The complex-float kernels use the coefficients rounded
to float; |G(k)|^2 - 1 of the rounded values bounds the norm change of one
sweep.  Kept as a0 = m (1 - 2 kappa) - 1, the rounding of the diagonal factor
no longer dominates.  (The rounding of the arithmetic itself is a separate,
smaller effect: see the summation order of the folded recurrences in the
kernels.)
"""
import numpy as np


def _fixed_point(kap, tau, iters=600):
    a0 = 1 + 2 * kap
    am, ap = tau - kap, -kap - tau
    c = 0
    for _ in range(iters):
        m = 1 / (a0 - am * c)
        c = ap * m
    return {"d": m * (1 - 2 * kap), "am": m * (kap - tau), "ap": m * (kap + tau),
            "al": -m * am, "be": -c}


def _f32(z):
    return complex(np.float32(z.real), np.float32(z.imag))


def _max_gain(h, dt, omega, us, diff_form=True):
    k = np.linspace(0, np.pi, 600)
    e = np.exp(1j * k)
    worst = 0.0
    for u in us:
        cf = _fixed_point(1j * dt / (4 * h * h), dt * omega / (4 * h) * u)
        d = 1 + _f32(cf["d"] - 1) if diff_form else _f32(cf["d"])
        num = d + _f32(cf["am"]) / e + _f32(cf["ap"]) * e
        den = (1 - _f32(cf["al"]) / e) * (1 - _f32(cf["be"]) * e)
        exact = (cf["d"] + cf["am"] / e + cf["ap"] * e) / ((1 - cf["al"] / e) * (1 - cf["be"] * e))
        assert np.abs(np.abs(exact) - 1).max() < 1e-13
        worst = max(worst, float(np.abs(np.abs(num / den) ** 2 - 1).max()))
    return worst


def test_interior_gain_bounds_of_the_physics_grids():
    us = -6.4 + 0.05 * np.arange(257)  # y (x lines) and x (y lines) of the 256^2 grids
    xy = _max_gain(0.05, 1e-4, 0.8, us)
    z = _max_gain(0.025, 1e-4, 0.0, [0.0])
    assert xy < 3.6e-9 and z < 4.0e-9, (xy, z)
    # the per-step bounds of the physics tests: two sweeps per 2D step, three
    # per 3D step
    from tests.test_physics import NORM_PER_STEP_2D, NORM_PER_STEP_3D
    assert 2 * xy <= NORM_PER_STEP_2D and 2 * xy + z <= NORM_PER_STEP_3D


def test_diagonal_factor_rounded_whole_is_an_order_worse():
    us = -6.4 + 0.05 * np.arange(0, 257, 16)
    plain = _max_gain(0.05, 1e-4, 0.8, us, diff_form=False)
    diff = _max_gain(0.05, 1e-4, 0.8, us, diff_form=True)
    assert plain > 1e-8 and plain > 10 * diff, (plain, diff)
