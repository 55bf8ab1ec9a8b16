"""Dense-matrix forms of the discrete rotating-GP operators (test helper).

Built directly from the continuum operators of the paper (Sec. 2):
    H1 = V + g|psi|^2                         (Eq. eq1)
    H2 = -(1/2) d^2/dx^2 - i Omega y d/dx      (Eq. eq2)
    H3 = -(1/2) d^2/dy^2 + i Omega x d/dy      (Eq. eq3)
    H4 = -(1/2) d^2/dz^2                       (3D, "identical prescription")
with the 3-point second difference and the central first difference on the
interior points (Dirichlet zero edges), assembled by Kronecker products.  A
Crank-Nicolson substep over Delta is (1 + i Delta H/2) psi' = (1 - i Delta H/2)
psi in real time and (1 + Delta H/2) psi' = (1 - Delta H/2) psi in imaginary
time (Delta -> -i Delta).  This is an independent construction from the
tridiagonal coefficients of Eqs. eqD.11/eq5 that the oracle uses.
"""
from __future__ import annotations

import numpy as np


def _d2(n_int: int, h: float) -> np.ndarray:
    m = n_int - 1
    return (np.diag(-2.0 * np.ones(m)) + np.diag(np.ones(m - 1), 1)
            + np.diag(np.ones(m - 1), -1)) / h ** 2


def _d1(n_int: int, h: float) -> np.ndarray:
    m = n_int - 1
    return (np.diag(np.ones(m - 1), 1) - np.diag(np.ones(m - 1), -1)) / (2 * h)


def _coords(n_int: int, h: float) -> np.ndarray:
    return -0.5 * n_int * h + np.arange(1, n_int) * h


def _kron_axis(mats_by_axis, dim):
    """Kronecker product with x fastest: order (z, y, x)."""
    out = np.ones((1, 1))
    for a in reversed(range(dim)):
        out = np.kron(out, mats_by_axis[a])
    return out


class DenseOps:
    def __init__(self, n, h, gamma, nu, lam, g, omega):
        self.n, self.h, self.dim = tuple(n), tuple(h), len(n)
        self.g, self.omega = g, omega
        dim = self.dim
        eye = [np.eye(n[a] - 1) for a in range(dim)]
        xs = [_coords(n[a], h[a]) for a in range(dim)]

        def along(a, m):
            mats = list(eye)
            mats[a] = m
            return _kron_axis(mats, dim)

        self.X = along(0, np.diag(xs[0]))
        self.Y = along(1, np.diag(xs[1]))
        self.Dx = along(0, _d1(n[0], h[0]))
        self.Dy = along(1, _d1(n[1], h[1]))
        self.H2 = -0.5 * along(0, _d2(n[0], h[0])) - 1j * omega * self.Y @ self.Dx
        self.H3 = -0.5 * along(1, _d2(n[1], h[1])) + 1j * omega * self.X @ self.Dy
        self.Hz = -0.5 * along(2, _d2(n[2], h[2])) if dim == 3 else None
        pot = gamma ** 2 * np.diag(self.X) ** 2 + nu ** 2 * np.diag(self.Y) ** 2
        if dim == 3:
            Z = along(2, np.diag(xs[2]))
            pot = pot + lam ** 2 * np.diag(Z) ** 2
        self.V = 0.5 * pot
        self.Lz = 1j * (self.Y @ self.Dx - self.X @ self.Dy)
        kin = self.H2 + self.H3 + (self.Hz if dim == 3 else 0)
        # H2 + H3 already contain -Omega L_z
        self.Hlin = kin + np.diag(self.V)
        self.vol = float(np.prod(h))

    # interior <-> full (N+1)^d array
    def interior(self, psi_full: np.ndarray) -> np.ndarray:
        sl = tuple(slice(1, -1) for _ in range(self.dim))
        return psi_full[sl].reshape(-1)

    def full(self, v: np.ndarray) -> np.ndarray:
        shape = tuple(self.n[a] + 1 for a in reversed(range(self.dim)))
        out = np.zeros(shape, dtype=np.complex128)
        sl = tuple(slice(1, -1) for _ in range(self.dim))
        out[sl] = v.reshape(tuple(self.n[a] - 1 for a in reversed(range(self.dim))))
        return out

    def cn(self, H, v, dt, imag):
        z = dt if imag else 1j * dt
        eye = np.eye(H.shape[0])
        return np.linalg.solve(eye + 0.5 * z * H, (eye - 0.5 * z * H) @ v)

    def step(self, v, dt, imag):
        z = dt if imag else 1j * dt
        v = np.exp(-z * (self.V + self.g * np.abs(v) ** 2)) * v
        v = self.cn(self.H2, v, dt, imag)
        v = self.cn(self.H3, v, dt, imag)
        if self.dim == 3:
            v = self.cn(self.Hz, v, dt, imag)
        if imag:
            v = v / np.sqrt(self.vol * np.sum(np.abs(v) ** 2))
        return v
