"""FP64 CPU oracle for the Lippmann-Schwinger PSFD solver (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. It shares no code with the CUDA path: it
has its own discrete Fourier transforms (``fft.py``), its own stack
recursion, Green's function, Krylov solver and extraction, all in complex128.
"""
from .psfd_oracle import *  # noqa: F401,F403
from .isolated_oracle import *  # noqa: F401,F403
from .differential_oracle import *  # noqa: F401,F403
