"""GB300-native lattice Boltzmann solver for Maxwell-Stefan multicomponent
diffusion (MRT model of Chai, Guo, Wang and Shi, arXiv:1808.06787).

The compute path is the CUDA library ``_build/liblbms.so`` (sources in
``csrc/``, C ABI in ``include/lbms.h``); ``lbms`` binds it with ctypes and uses
PyTorch only for device memory and streams.
"""

from .lbms import (  # noqa: F401
    EXPORTED,
    BatchSolver,
    LbmsError,
    Solver,
    lbms_create,
    lbms_destroy,
    lbms_gradient,
    lbms_last_error,
    lbms_mass,
    lbms_moments,
    lbms_set_boundary,
    lbms_set_state,
    lbms_status,
    lbms_step,
    lbms_steps_done,
    lbms_workspace_size,
    load,
)
from .autograd import MaxwellStefanLB, RunSpec, simulate  # noqa: F401
from .slab import DistSlabSolver, SlabSolver  # noqa: F401
from . import scenarios  # noqa: F401
