"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the oracle.

This package holds input generation only: meshes of the meridian (z, rho) half-plane,
particle samplers and initial field values.  None of the PIC method's arithmetic
(Whitney forms, Hodge matrices, SPAI, push, walk, scatter) lives here; both the oracle
and the GPU library derive everything from the raw arrays produced here.

Array conventions used by every generator:

* ``nodes``   float64 (N0, 2): columns (z, rho), rho >= 0.
* ``tris``    int32   (N2, 3): node indices, counter-clockwise in the (z, rho) frame.
* ``bedges``  int32   (Nb, 2): node pairs of every mesh boundary edge.
* ``btags``   int32   (Nb,):   BC_PEC, BC_AXIS or BC_ABSORB.
"""

BC_PEC = 1      # conducting wall: tangential E = 0, particles absorbed
BC_AXIS = 2     # symmetry axis rho = 0: natural (PMC) field BC, particles kept
BC_ABSORB = 3   # open port: natural field BC, particles absorbed

from .meshes import (  # noqa: E402
    jittered_delaunay, rect_mesh, cavity_mesh, bwo_mesh, bwo_small_mesh, bwo_wall, diode_mesh,
    two_triangle_mesh, four_triangle_mesh,
)
from .particles import (  # noqa: E402
    uniform_in_volume_rect, bwo_beam, uniform_in_mesh, maxwellian, cavity_particles,
)
from .fields import tm0np_edge_dofs, tm0np_omega, random_edge_values  # noqa: E402
from .cavity import cavity_workload, cavity_weight, cavity_modes  # noqa: E402
