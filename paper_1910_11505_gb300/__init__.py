"""GB300-native solver for the stochastic Galerkin diffusion system of arXiv 1910.11505.

The compute path lives in the CUDA library built from ``csrc/`` (C ABI in ``include/sg.h``);
``sg`` is its ctypes binding and ``workloads`` holds the seeded synthetic inputs.
"""

from . import sg  # noqa: F401
from .sg import (  # noqa: F401
    SGError, SGHandle, sg_default_params, sg_dims, sg_export, sg_free, sg_gmres_solve,
    sg_launch_count, sg_matvec, sg_matvec_lowp, sg_nnz, sg_params, sg_precond_apply, sg_rhs,
    sg_setup, load_library,
)
