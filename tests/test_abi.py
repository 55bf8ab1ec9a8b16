"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point that include/rotgp.h declares (no compute calls)."""
import ctypes
import os
import re

import pytest

from paper_1906_06327_gb300 import build as rbuild
from paper_1906_06327_gb300 import rotgp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "rotgp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rotgp_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_binding_exports():
    assert sorted(rotgp.EXPORTS) == _declared()


def test_library_builds_loads_and_exports_every_symbol():
    path = rbuild.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_create_error_message_without_work():
    """Argument validation happens before any CUDA call."""
    lib = rotgp.load()
    grid = rotgp.Grid(4, (ctypes.c_int * 3)(8, 8, 8), (ctypes.c_double * 3)(0.1, 0.1, 0.1))
    phys = rotgp.Phys(1, 1, 1, 0, 0, 1e-3)
    h = ctypes.c_void_p()
    rc = lib.rotgp_create(ctypes.byref(grid), ctypes.byref(phys), 1, None, ctypes.byref(h))
    assert rc == rotgp.ROTGP_EINVAL
    assert b"dim" in lib.rotgp_last_error(None)
    grid = rotgp.Grid(2, (ctypes.c_int * 3)(8, 3, 0), (ctypes.c_double * 3)(0.1, 0.1, 0))
    rc = lib.rotgp_create(ctypes.byref(grid), ctypes.byref(phys), 1, None, ctypes.byref(h))
    assert rc == rotgp.ROTGP_EINVAL
    grid = rotgp.Grid(2, (ctypes.c_int * 3)(8, 8, 0), (ctypes.c_double * 3)(0.1, 0.1, 0))
    bad = rotgp.Phys(1, 1, 1, 0, 0, -1.0)
    rc = lib.rotgp_create(ctypes.byref(grid), ctypes.byref(bad), 1, None, ctypes.byref(h))
    assert rc == rotgp.ROTGP_EINVAL
    rc = lib.rotgp_create(ctypes.byref(grid), ctypes.byref(phys), 7, None, ctypes.byref(h))
    assert rc == rotgp.ROTGP_EINVAL


def test_ptxas_reports_no_spills_in_fp32_sweeps():
    """The complex-float imaginary-time sweep kernels (the bandwidth-bound hot
    path) keep their working set in registers and shared memory (at most a
    word or two spilled)."""
    rbuild.build()
    path = os.path.join(rbuild.BUILD, "ptxas.log")
    if not os.path.exists(path):
        pytest.skip("library was not built in this tree; no ptxas log")
    log = open(path).read()
    blocks = re.findall(r"Function properties for (\S+)\n\s+(\d+) bytes stack frame, "
                        r"(\d+) bytes spill stores", log)
    # mangled names: k_sweep_strided<float, V, C, REDUCE>, k_sweep_x<float, V, C, IMAG, VEC16>
    hot = [(f, int(sp)) for f, _, sp in blocks
           if ("k_sweep_strided" in f and "IfLi" in f)
           or ("k_sweep_x" in f and "IfLi" in f and re.search(r"ELb1ELb[01]E", f))]
    assert len(hot) >= 8
    assert all(sp <= 16 for _, sp in hot), hot
