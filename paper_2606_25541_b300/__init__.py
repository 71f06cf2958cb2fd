"""B300-native Lippmann-Schwinger PSFD solver for EUV mask scattering.

The compute path is the CUDA library ``libpsfd.so`` behind the C ABI declared in
``include/psfd.h``; :mod:`paper_2606_25541_b300.psfd` is its thin ctypes binding and
:mod:`paper_2606_25541_b300.layouts` generates seeded synthetic workloads.
Importing the package does not load the library; the first binding call does, and
raises if it has not been built.
"""
__all__ = ["layouts"]
