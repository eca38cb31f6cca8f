"""GB300-native dense Krylov solvers (CG, restarted GMRES, mixed-precision
refinement, batched and served solves) behind a C ABI (``include/ls.h``).

The CUDA library is loaded lazily by :mod:`paper_1511_07207_gb300.binding`;
importing this package alone does not touch the GPU.
"""
__all__ = ["binding", "inputs"]
