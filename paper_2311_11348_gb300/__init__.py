"""GB300 (sm_103a) solver for the quadrature-free, p-adaptive DG shallow water
scheme of Faghih-Naini et al. (2023).

The compute path is the CUDA library ``libswedg`` (``csrc/``), reached through
the thin ctypes binding in ``swedg.py``; ``inputs.py`` makes seeded synthetic
workloads.  Importing the package does not load the library; ``swedg.load()``
does, and fails loudly when the library is missing.
"""
__all__ = ["inputs", "swedg"]
