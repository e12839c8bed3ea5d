"""Batched ripple sweep: seeded backward-wave-oscillator instances and their union.

Instance i draws from its own seed: ripple depth 0.2-0.6 cm, period 1.4-2.0 cm, 8-16
periods, beam 300-500 kV and 1-5 kA, a mesh of 20k-80k triangles.  All instances share
the wall's mean radius (1.5 cm), 2 cm guides, the guide field and the macro-particle
weight; an instance's particle count is its beam charge in the ripple section over that
weight, kept within 0.5M-4M (the charge a clipped count carries sets the instance's
effective current).  The annular beam (0.1 cm thick) sits at 70% of the narrowest wall
radius.

The instances are batched by ``paper_1701_03784_gb300.batch.union`` (re-exported here):
side by side along z, one simulation of the union advances all of them.
"""
import math

import numpy as np

from paper_1701_03784_gb300.batch import union  # noqa: F401  (the sweep's batching)

from .meshes import bwo_mesh, bwo_wall
from .particles import bwo_beam

QE = 1.602176634e-19
C0 = 299792458.0
MC2_VOLTS = 510998.95
R0 = 1.5e-2
GUIDE = 2e-2
N_MIN, N_MAX = 500_000, 4_000_000
# common macro-particle weight: a 3 kA, 12 x 1.7 cm, 400 kV beam in 2M particles
WEIGHT = 3e3 * 12 * 1.7e-2 / (0.8279 * C0) / (QE * 2_000_000)


def sweep_params(i):
    """Parameters of instance i (seeded by i)."""
    rng = np.random.default_rng(i)
    return dict(depth=rng.uniform(0.2e-2, 0.6e-2), period=rng.uniform(1.4e-2, 2.0e-2),
                n_periods=int(rng.integers(8, 17)), voltage=rng.uniform(300e3, 500e3),
                current=rng.uniform(1e3, 5e3), n_tri=int(rng.integers(20_000, 80_001)))


def sweep_particles(i, scale=1.0):
    """Particle count of instance i: its beam charge in the slow-wave section over the
    common weight, clipped to [N_MIN, N_MAX], times scale."""
    p = sweep_params(i)
    zs0, zs1 = bwo_wall(r0=R0, ripple=p["depth"], period=p["period"],
                        n_periods=p["n_periods"], guide=GUIDE)[2]
    gamma = 1.0 + p["voltage"] / MC2_VOLTS
    vz = C0 * math.sqrt(1.0 - 1.0 / gamma ** 2)
    charge = p["current"] * (zs1 - zs0) / vz
    n = int(min(max(round(charge / (QE * WEIGHT)), N_MIN), N_MAX))
    return max(1, int(round(n * scale)))


def sweep_instance(i, scale=1.0, mesh_scale=1.0, tri_per_cm2=None):
    """Mesh and beam of instance i.  ``scale`` multiplies the particle count and
    ``mesh_scale`` the triangle count (tests and surrogate data use fractions of them);
    ``tri_per_cm2``, if given, sets the triangle count from the meridian area instead, so
    that every instance has the same mesh spacing (the surrogate's data: the drawn count
    would otherwise be a hidden input)."""
    p = sweep_params(i)
    n_tri = max(2000, int(p["n_tri"] * mesh_scale))
    if tri_per_cm2 is not None:
        R, z_end, _ = bwo_wall(r0=R0, ripple=p["depth"], period=p["period"],
                               n_periods=p["n_periods"], guide=GUIDE)
        zz = np.linspace(0.0, z_end, 20001)
        area_cm2 = float(np.trapezoid(R(zz), zz)) * 1e4
        n_tri = max(2000, int(round(tri_per_cm2 * area_cm2)))
    # deep, short ripples on a coarse mesh need the wall sampled more finely to conform
    for refine in (1.0, 0.7, 0.5, 0.35):
        try:
            nodes, tris, be, bt = bwo_mesh(n_tri, seed=3000 + i, wall_refine=refine, r0=R0,
                                           ripple=p["depth"], period=p["period"],
                                           n_periods=p["n_periods"], guide=GUIDE)
            break
        except RuntimeError:
            if refine == 0.35:
                raise
    R, z_end, (zs0, zs1) = bwo_wall(r0=R0, ripple=p["depth"], period=p["period"],
                                    n_periods=p["n_periods"], guide=GUIDE)
    gamma = 1.0 + p["voltage"] / MC2_VOLTS
    vz = C0 * math.sqrt(1.0 - 1.0 / gamma ** 2)
    n = sweep_particles(i, scale)
    rb = 0.7 * (R0 - p["depth"])
    z, r, ur, up, uz = bwo_beam(n, r_in=rb - 0.05e-2, r_out=rb + 0.05e-2, z0=zs0, z1=zs1,
                                voltage=p["voltage"], seed=4000 + i)
    return dict(params=p, nodes=nodes, tris=tris, be=be, bt=bt, z_end=z_end, r_out=R0, z=z, r=r,
                ur=ur, up=up, uz=uz, n=n, sws=(zs0, zs1), vz=vz,
                current_eff=n * QE * WEIGHT * vz / (zs1 - zs0))


SURROGATE_SCALE = 0.05
SURROGATE_TRI_PER_CM2 = 450.0


def surrogate_instance(i):
    """Instance i as the surrogate's data takes it: 450 triangles per cm^2 of the meridian
    plane (the same spacing, ~0.7 mm, for every instance) and SURROGATE_SCALE of its
    particles."""
    return sweep_instance(i, scale=SURROGATE_SCALE, tri_per_cm2=SURROGATE_TRI_PER_CM2)
