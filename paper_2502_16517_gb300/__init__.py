"""GB300-native SPH view path: field-selective AoS->SoA views fused with cell-linked-list density and force
loops, behind the C-ABI library ``libsph`` (declared in ``include/sph.h``).

Importing the package loads nothing.  ``paper_2502_16517_gb300.sph`` is the ctypes binding of the library and
raises when the compiled library is missing; ``paper_2502_16517_gb300.workloads`` makes seeded inputs.
"""
__all__ = ["sph", "workloads", "build"]
