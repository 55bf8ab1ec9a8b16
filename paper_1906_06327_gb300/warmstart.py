"""Learned warm start: data from the solver, training and evaluation.

The network (``rotgp_ws_*`` in the CUDA library) proposes the initial wave
function of a 2D rotating run from its parameters (Omega, g, nu).  Its
training set is made by the solver itself: many instances of one grid,
started from the same seeded one-vortex state of Eq. fun and propagated in
imaginary time with the persistent batch step until converged (or for a
fixed budget).  The evaluation then runs imaginary time to convergence from
three starts for each held-out parameter set, as Sec. 3 compares starts:
the analytic seeded start, the network's proposal, and a lattice converged
beforehand at a lower Omega (the paper's practice, Sec. 1 and Sec. 3).
Every numerical step runs in the CUDA library; this module orders the calls.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from .rotgp import Batch, WarmStart


@dataclass(frozen=True)
class Setup:
    """The runs of the warm-start workload: G x G intervals on [-L, L]^2,
    gamma = 1, imaginary-time step dt, seeded start `seed`."""
    grid: int = 128
    half_width: float = 12.0
    dt: float = 1e-3
    seed: int = 5

    @property
    def h(self) -> float:
        return 2.0 * self.half_width / self.grid

    @property
    def window(self) -> int:
        """Steps per convergence check: one time unit."""
        return max(1, int(round(1.0 / self.dt)))

    def spec(self, omega, g, nu) -> dict:
        return dict(n=(self.grid, self.grid), h=(self.h, self.h), gamma=1.0, nu=float(nu),
                    g=float(g), omega=float(omega), dt=self.dt)


def converge(setup: Setup, prm, starts=None, rel_tol=1e-6, max_units=400, stream=0):
    """Imaginary time to convergence for each parameter set (|mu(t) -
    mu(t - 1)| <= rel_tol |mu(t)| over one time unit, vortex count
    unchanged), all in one batch with the persistent step.  starts: None
    (the seeded analytic start) or ABI wave functions to load (normalised).
    Returns (states, observables, steps, converged flags, wall seconds)."""
    prm = np.asarray(prm, dtype=np.float64).reshape(-1, 3)
    b = Batch([setup.spec(*p) for p in prm], stream=stream)
    for i, inst in enumerate(b.instances):
        if starts is None:
            inst.init_analytic(1, seed=setup.seed)
        else:
            inst.set_psi(np.ascontiguousarray(starts[i], dtype=np.complex128), normalise=True)
    b.sync()
    t0 = time.perf_counter()
    steps, conv = b.converge(rel_tol, setup.window, max_units * setup.window, mode="persistent")
    b.sync()
    wall = time.perf_counter() - t0
    obs = b.observables()
    states = np.stack([inst.get_psi() for inst in b.instances])
    b.close()
    return states, obs, np.asarray(steps), np.asarray(conv), wall


def train(ws: WarmStart, setup: Setup, prm, states, epochs=200, batch=16, lr=1e-3, seed=0):
    """Adam on the mean squared error between the network's outputs and
    2 L psi of the converged states; returns the loss of every step."""
    prm = np.asarray(prm, dtype=np.float64).reshape(-1, 3)
    n = prm.shape[0]
    rng = np.random.default_rng(seed)
    losses = []
    for ep in range(epochs):
        order = rng.permutation(n)
        # cosine decay of the learning rate over the epochs
        lr_ep = 0.5 * lr * (1.0 + np.cos(np.pi * ep / epochs))
        for s in range(0, n - batch + 1, batch):
            idx = order[s:s + batch]
            losses.append(ws.train_step(prm[idx], setup.half_width,
                                        np.ascontiguousarray(states[idx]), max(lr_ep, 1e-5)))
    return np.asarray(losses)


def lower_omega(prm, delta=0.1):
    """The parameter sets of the pre-calculated starts: Omega - delta."""
    q = np.array(prm, dtype=np.float64).reshape(-1, 3)
    q[:, 0] -= delta
    return q


def evaluate(ws: WarmStart, setup: Setup, prm, lower=0.1, stream=0) -> dict:
    """Imaginary time to convergence for each parameter set from three starts:
    the analytic seeded start of Eq. fun, the network's proposal times the
    same random phase, and the lattice converged beforehand at Omega - lower
    (the pre-calculated start of the paper; its own convergence is not
    counted).  Per start: steps, converged flags, mu, E, vortex counts and
    the wall time of the batch."""
    prm = np.asarray(prm, dtype=np.float64).reshape(-1, 3)
    out = {}
    starts = {"analytic": None,
              "learned": ws.propose(prm, setup.half_width, seed=setup.seed)}
    if lower:
        starts["lower_omega"] = converge(setup, lower_omega(prm, lower), stream=stream)[0]
    for name, st in starts.items():
        _, obs, steps, conv, wall = converge(setup, prm, starts=st, stream=stream)
        out[name] = {"steps": steps, "converged": conv, "wall_s": wall,
                     "mu": np.array([o["mu"] for o in obs]),
                     "energy": np.array([o["energy"] for o in obs]),
                     "vortices": np.array([o["vortices"] for o in obs])}
    return out
