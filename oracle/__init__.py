"""FP64 CPU oracle of the staggered-grid Navier-Stokes time step.

TEST INFRASTRUCTURE ONLY: used by tests/, the smoke check and the CPU-baseline
leg of bench.py.  It shares no code with the CUDA library.
"""
from .oracle import (Oracle, bc_faces, build, compile_sources, exact_poisson_periodic,  # noqa: F401
                     load_library, set_threads, source_paths, PERIODIC, WALL)
