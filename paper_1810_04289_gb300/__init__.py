"""GB300 (sm_103a) monolithic fluid-structure Newton-Krylov-Schwarz solver.

The solver is the CUDA library built from csrc/ behind the C ABI of
include/fsi.h; `fsi` is its Python binding. Importing the package does not load
the library; importing `paper_1810_04289_gb300.fsi` and calling any entry point
does, and fails loudly if it has not been built.
"""
__all__ = ["fsi", "build"]
