"""The single backward-wave-oscillator workload: rippled slow-wave structure, annular beam.

SI units.  Wall R(z) = 1.5 cm + 0.4 cm sin(2 pi z / 1.67 cm) over 12 periods with 3 cm
straight guides (~200k triangles); beam annulus rho in [0.85, 0.95] cm over the ripple
section, 400 kV, 3 kA, thermal spread 1e-3 u_z; guide field B_z = 2.5 T; seeded random
edge fields at 1e-3 of the beam's self-field scale; time step 8.8e-14 s (half the SPAI
leapfrog limit of this mesh, 1.77e-13 s).
"""
import math

import numpy as np

from .meshes import bwo_mesh, bwo_wall
from .particles import bwo_beam
from .fields import random_edge_values

EPS0 = 8.8541878128e-12
MU0 = 1.25663706212e-6
C0 = 299792458.0
QE = -1.602176634e-19
ME = 9.1093837015e-31
DT_BWO = 8.8e-14
BZ_BWO = 2.5


def bwo_workload(n_particles, seed=2002, n_tri=200_000, mesh_seed=1002):
    nodes, tris, be, bt = bwo_mesh(n_tri, seed=mesh_seed)
    R, z_end, (zs0, zs1) = bwo_wall()
    z, r, ur, up, uz = bwo_beam(n_particles, z0=zs0, z1=zs1, voltage=400e3, seed=seed)
    gamma = 1.0 + 400e3 / 510998.95
    vz = C0 * math.sqrt(1.0 - 1.0 / gamma ** 2)
    # beam charge in the ripple section, I L / v_z, shared by the macro-particles
    weight = 3e3 * (zs1 - zs0) / vz / (abs(QE) * n_particles)
    # self-field scale of the beam, E ~ lambda / (2 pi eps0 rho)
    e_scale = 1e-3 * (3e3 / vz) / (2 * math.pi * EPS0 * 0.9e-2)
    return dict(nodes=nodes, tris=tris, be=be, bt=bt, z=z, r=r, ur=ur, up=up, uz=uz,
                weight=weight, e_scale=e_scale, bz=BZ_BWO, dt=DT_BWO)


def bwo_edge_field(n_edges, e_scale, seed=7):
    """Seeded edge DOFs: E ~ e_scale times a mean edge length of 2e-4 m."""
    return random_edge_values(n_edges, e_scale * 2e-4, seed)
