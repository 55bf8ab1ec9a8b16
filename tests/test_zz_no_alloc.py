"""rotgp_observables_noalloc: the allocation-free observables entry point.

It serves callers that cannot call cudaMalloc (device memory owned by
another allocator, a fixed memory budget, loops that must not add the
synchronisation of an allocation).  Checked through the C ABI against the
context's rotgp_observables on the same state, on two calls in a row, with
the tolerances of the other parity tests.  Kept in its own file, collected
last.
"""
import ctypes

import numpy as np
import pytest

from paper_1906_06327_gb300 import inputs
from paper_1906_06327_gb300 import rotgp

pytestmark = pytest.mark.gpu

KEYS = ("norm", "mu", "energy", "mu_c", "energy_c", "rms_x", "rms_y", "rms_z", "rms_r",
        "max_density", "mu4", "energy4")


@pytest.mark.parametrize("n,h,precision,tol", [
    ((64, 48), (0.2, 0.25), "fp64", 1e-12),
    ((40, 36, 22), (0.3, 0.3, 0.25), "fp64", 1e-12),
    ((96, 80), (0.12, 0.15), "fp32", 2e-6),
    ((48, 40, 36), (0.25, 0.25, 0.2), "fp32", 2e-6),
])
def test_noalloc_observables_match_context_twice(n, h, precision, tol):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    phys = dict(gamma=1.0, nu=1.1, lam=1.4, g=80.0, omega=0.6, dt=1e-3)
    s = rotgp.Solver(n, h, precision=precision, **phys)
    s.init_analytic(1, inputs.random_phase_field(n[0], n[1], 3), 1.0, 0.9)
    s.step_imag(40)
    ref = s.observables()
    dtype = torch.complex128 if precision == "fp64" else torch.complex64
    psi = torch.zeros(s.shape, dtype=dtype, device="cuda")
    s.get_psi(psi)
    torch.cuda.synchronize()
    lib = rotgp.load()
    dim = len(n)
    grid = rotgp.Grid(dim, (ctypes.c_int * 3)(*(list(n) + [0] * (3 - dim))),
                      (ctypes.c_double * 3)(*(list(h) + [0.0] * (3 - dim))))
    cphys = rotgp.Phys(phys["gamma"], phys["nu"], phys["lam"], phys["g"], phys["omega"],
                       phys["dt"])
    prec = rotgp.ROTGP_FP64 if precision == "fp64" else rotgp.ROTGP_FP32
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = rotgp.Obs()
        rc = lib.rotgp_observables_noalloc(ctypes.byref(grid), ctypes.byref(cphys), prec,
                                           ctypes.c_void_p(psi.data_ptr()),
                                           ctypes.c_void_p(stream), ctypes.byref(out))
        assert rc == rotgp.ROTGP_OK, lib.rotgp_last_error(None)
        got = out.as_dict()
        for k in KEYS:
            assert abs(got[k] - ref[k]) <= tol * max(abs(ref[k]), 1e-300), (call, k, got[k], ref[k])
        assert got["vortices"] == -1 and got["step"] == 0
        assert got["flags"] == ref["flags"]
    # the Python helper goes through the same entry point
    again = rotgp.observables_noalloc(n, h, psi, gamma=phys["gamma"], nu=phys["nu"],
                                      lam=phys["lam"], g=phys["g"], omega=phys["omega"],
                                      stream=stream)
    assert abs(again["energy"] - ref["energy"]) <= tol * abs(ref["energy"])


def test_noalloc_rejects_grids_beyond_the_fixed_scratch():
    lib = rotgp.load()
    grid = rotgp.Grid(3, (ctypes.c_int * 3)(512, 512, 200), (ctypes.c_double * 3)(0.1, 0.1, 0.1))
    phys = rotgp.Phys(1, 1, 1, 0, 0, 1e-3)
    out = rotgp.Obs()
    rc = lib.rotgp_observables_noalloc(ctypes.byref(grid), ctypes.byref(phys), rotgp.ROTGP_FP32,
                                       ctypes.c_void_p(1 << 20), None, ctypes.byref(out))
    assert rc == rotgp.ROTGP_EINVAL
    assert b"at most 33554432" in lib.rotgp_last_error(None)
