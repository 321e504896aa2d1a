"""GB300-native explicit staggered-grid Navier-Stokes time step.

The compute path is libgb300cfd.so (hand-written sm_103a CUDA behind a C ABI,
declared in include/gb300cfd.h); this package is its thin Python binding.
"""
from ._lib import CfdError, lib, library_path  # noqa: F401
from .grid import (Grid, mask, U, V, W, P, WU, WV, WW, U1, V1, W1, P2, R,  # noqa: F401
                   LU, LV, LW, LP, SET_U, SET_W, SET_U1, PERIODIC, WALL)
from .autograd import Rollout  # noqa: F401
from .descriptor import Descriptor, GeneratedKernel  # noqa: F401
