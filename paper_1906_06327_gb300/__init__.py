"""GB300-native split-step Crank-Nicolson solver for the rotating
Gross-Pitaevskii equation (Kumar et al., Sec. 2).

The numerics run in the CUDA library ``librotgp.so`` behind the C ABI
declared in ``include/rotgp.h``; ``rotgp`` is a thin ctypes binding to it and
``inputs`` the seeded input generators.  Importing this package does not load
the library; the first call into ``rotgp`` does, and fails loudly if it is
missing.
"""
__all__ = ["rotgp", "inputs"]
