"""B300-native CHFPE hot path (arXiv 2509.25840): RK4 propagation of the classical hierarchical
Fokker-Planck equations on a uniform (q,p) grid, optical insertions and phase-space reductions,
behind the C-ABI library ``libchfpe.so`` (declared in ``include/chfpe.h``).

Importing the package loads nothing; ``paper_2509_25840_b300.chfpe`` loads the CUDA library and
fails loudly if it is missing.
"""
__all__ = ["inputs", "chfpe"]
