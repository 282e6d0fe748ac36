"""GB300 pseudopotential D2Q9 lattice Boltzmann step with the shaped ("Smooth C-S")
equation of state.

The compute path is the CUDA library ``libpplbm.so`` (include/pplbm.h) behind a
ctypes binding; PyTorch provides device memory and streams only. Nothing here
computes the method on the CPU: if the library is missing, import of the
simulation class fails.
"""
from ._lib import (BC_PERIODIC, BC_PERIODIC_X, BC_PERIODIC_Y, BC_WALL_BOTTOM, BC_WALL_TOP, BC_WALLS_Y,  # noqa: F401
                   EOS_CS, EOS_SMOOTH, EOS_PENG, EOS_SMOOTH_MOD, FORCING_GUO, FORCING_LI, RELAX_MRT, RELAX_TWO_PHASE, PPLBMError,
                   lib)
from ._lib import PLAN_GRAPH, PLAN_LAUNCHES, PLAN_PERSISTENT, PLAN_PIPELINED  # noqa: F401
from .batch import Batch  # noqa: F401
from .fd import FDSolver  # noqa: F401
from .lattice import EOSParams, Relax, Simulation, eos_setup  # noqa: F401
