"""The arithmetic behind the complex-float real-time kernels, checked on the
CPU by emulating float32 with single-rounding FMAs (numpy: exact products in
double, one rounding to float32).

One real-time split step along x lines: H1 (Eq. eq1) as the rotation
exp(-i theta) = 1 + c1 - i s1, then the folded Thomas solve of Eqs.
eqD.9-eqD.11 (forward d' = (1 + a0) w + am w_- + ap w_+ + al d', backward
x = d' + be x_+, a0 kept as its difference from 1).  Two orders of the same
arithmetic:

* rounded: the rotated point w rounded on its own, each recurrence step
  rounding its small terms into the O(1) value one FMA at a time;
* carried (the kernels' order): w = v + dl with the increment dl carried
  into the forward sum, small terms summed first, the O(1) value added once.

Exact arithmetic keeps the norm.  In float the first order gains norm
steadily (the second-order part of a small rotation is lost whenever a
component of v passes an extremum, and each rounding into the large value
adds a small bias); the second does not.
"""
import numpy as np

F, D = np.float32, np.float64


def _fixed_point(kap, tau, iters=200):
    a0 = 1 + 2 * kap
    am, ap = tau - kap, -kap - tau
    c = 0
    for _ in range(iters):
        m = 1 / (a0 - am * c)
        c = ap * m
    return {"d": m * (1 - 2 * kap) - 1, "am": m * (kap - tau), "ap": m * (kap + tau),
            "al": -m * am, "be": -c}


def _fma(a, b, c):
    return (np.asarray(a, D) * np.asarray(b, D) + np.asarray(c, D)).astype(F)


def _cfma(k, br, bi, cr, ci):
    kr, ki = k
    return _fma(-ki, bi, _fma(kr, br, cr)), _fma(ki, br, _fma(kr, bi, ci))


def _norm_gain_per_step(order, N=128, L=16, h=0.05, dt=1e-4, steps=500):
    x = (-N / 2 + np.arange(N + 1)) * h
    ys = np.linspace(-1.5, 1.5, L)
    V = (x[None, :] ** 2 / 2 + ys[:, None] ** 2 / 2).astype(F)
    psi = np.exp(-x ** 2 / 2)[None, :] * np.ones((L, 1))
    psi[:, 0] = psi[:, -1] = 0
    re, im = psi.astype(F), np.zeros((L, N + 1), F)
    k = {n: (F(v.real), F(v.imag)) for n, v in _fixed_point(1j * dt / (4 * h * h), 0.0).items()}
    half = ((F(dt) * V).astype(F) * F(0.5)).astype(F)
    sh, ch = np.sin(half.astype(D)).astype(F), np.cos(half.astype(D)).astype(F)
    c1, s1 = ((F(-2) * sh) * sh).astype(F), ((F(2) * sh) * ch).astype(F)
    zero = np.zeros(L, F)
    n0 = (re.astype(D) ** 2 + im.astype(D) ** 2).sum()
    for _ in range(steps):
        if order == "rounded":
            wr, wi = _fma(c1, re, _fma(s1, im, re)), _fma(c1, im, _fma(-s1, re, im))
        else:
            dr, di = _fma(c1, re, (s1 * im).astype(F)), _fma(c1, im, (-s1 * re).astype(F))
            wr, wi = (re + dr).astype(F), (im + di).astype(F)
        out_r, out_i = np.zeros_like(re), np.zeros_like(re)
        pr, pi, qr, qi = zero, zero, zero, zero
        for p in range(1, N):
            if order == "rounded":
                sr, si = _cfma(k["d"], wr[:, p], wi[:, p], wr[:, p], wi[:, p])
            else:
                sr, si = _cfma(k["d"], wr[:, p], wi[:, p], dr[:, p], di[:, p])
            sr, si = _cfma(k["am"], pr, pi, sr, si)
            sr, si = _cfma(k["ap"], wr[:, p + 1], wi[:, p + 1], sr, si)
            sr, si = _cfma(k["al"], qr, qi, sr, si)
            if order != "rounded":
                sr, si = (re[:, p] + sr).astype(F), (im[:, p] + si).astype(F)
            out_r[:, p], out_i[:, p] = sr, si
            qr, qi, pr, pi = sr, si, wr[:, p], wi[:, p]
        zr, zi = zero, zero
        for p in range(N - 1, 0, -1):
            if order == "rounded":
                zr, zi = _cfma(k["be"], zr, zi, out_r[:, p], out_i[:, p])
            else:
                tr, ti = _cfma(k["be"], zr, zi, zero, zero)
                zr, zi = (out_r[:, p] + tr).astype(F), (out_i[:, p] + ti).astype(F)
            out_r[:, p], out_i[:, p] = zr, zi
        re, im = out_r, out_i
    return ((re.astype(D) ** 2 + im.astype(D) ** 2).sum() - n0) / n0 / steps


def test_rounding_order_decides_the_real_time_norm():
    rounded = _norm_gain_per_step("rounded")
    carried = _norm_gain_per_step("carried")
    assert rounded > 3e-9, rounded
    assert abs(carried) < 1e-9, carried
    assert rounded > 10 * abs(carried), (rounded, carried)
