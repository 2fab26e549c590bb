"""GB300-native preconditioned inexact interior-point QP solver (Karim & Solomonik).

The solver is the CUDA library ``libpcgipm.so`` (C ABI in include/pcgipm.h);
``paper_2104_12916_gb300.binding`` is its ctypes binding with the same call
names.  Importing this package does not load the library; the binding loads it
on first use and raises if it has not been built (``build.build()``).
"""
__all__ = ["binding", "build"]
