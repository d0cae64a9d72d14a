"""Seeded synthetic inputs for the VANSE lattice Boltzmann problem.

This package builds geometry flags, porosity fields and parameter sets.  It is
shared by the FP64 oracle and by the CUDA path, so it deliberately contains none
of the method's arithmetic: no moments, equilibria, boundary reconstruction,
unit conversion or viscosity law.  It only voxelises shapes, draws seeded random
fields and lists the physical parameters of each workload.
"""

from .geometry import (  # noqa: F401
    SOLID,
    FLUID,
    INLET,
    OUTLET,
    pipe_flags,
    aneurysm_flags,
    sac_mask,
    channel_flags,
    periodic_box_flags,
)
from .porosity import (  # noqa: F401
    coil_packings,
    coil_shape_tensor,
    plug_porosity,
    sac_random_porosity,
    wire_coil,
    wire_coil_order,
)
from .configs import (  # noqa: F401
    Problem,
    pipe_problem,
    aneurysm_problem,
    COIL_PHI_MIN,
    COIL_WINDOW,
    coil_problem,
    channel_problem,
    periodic_box_problem,
    WORKLOAD_CY,
    ANEURYSM_LAMBDA,
    PAPER_TABLE1,
)
