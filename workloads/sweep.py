"""Batched ripple sweep: seeded backward-wave-oscillator instances and their union.

Instance i draws from its own seed: ripple depth 0.2-0.6 cm, period 1.4-2.0 cm, 8-16
periods, beam 300-500 kV and 1-5 kA, a mesh of 20k-80k triangles.  All instances share
the wall's mean radius (1.5 cm), 2 cm guides, the guide field and the macro-particle
weight; an instance's particle count is its beam charge in the ripple section over that
weight, kept within 0.5M-4M (the charge a clipped count carries sets the instance's
effective current).  The annular beam (0.1 cm thick) sits at 70% of the narrowest wall
radius.

The union places the instances side by side along z (each shifted by the lengths of the
ones before it plus a 1 cm gap), so that one simulation of the union advances all of them:
every operator of the method is local to a mesh, and the union's meshes share no node.
"""
import math

import numpy as np

from .meshes import bwo_mesh, bwo_wall
from .particles import bwo_beam

QE = 1.602176634e-19
C0 = 299792458.0
MC2_VOLTS = 510998.95
R0 = 1.5e-2
GUIDE = 2e-2
GAP = 1e-2
N_MIN, N_MAX = 500_000, 4_000_000
# common macro-particle weight: a 3 kA, 12 x 1.7 cm, 400 kV beam in 2M particles
WEIGHT = 3e3 * 12 * 1.7e-2 / (0.8279 * C0) / (QE * 2_000_000)


def sweep_params(i):
    """Parameters of instance i (seeded by i)."""
    rng = np.random.default_rng(i)
    return dict(depth=rng.uniform(0.2e-2, 0.6e-2), period=rng.uniform(1.4e-2, 2.0e-2),
                n_periods=int(rng.integers(8, 17)), voltage=rng.uniform(300e3, 500e3),
                current=rng.uniform(1e3, 5e3), n_tri=int(rng.integers(20_000, 80_001)))


def sweep_instance(i, scale=1.0):
    """Mesh and beam of instance i.  ``scale`` multiplies the particle count (tests use
    small fractions of it)."""
    p = sweep_params(i)
    # deep, short ripples on a coarse mesh need the wall sampled more finely to conform
    for refine in (1.0, 0.7, 0.5, 0.35):
        try:
            nodes, tris, be, bt = bwo_mesh(p["n_tri"], seed=3000 + i, wall_refine=refine, r0=R0,
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
    charge = p["current"] * (zs1 - zs0) / vz
    n = int(min(max(round(charge / (QE * WEIGHT)), N_MIN), N_MAX))
    n = max(1, int(round(n * scale)))
    rb = 0.7 * (R0 - p["depth"])
    z, r, ur, up, uz = bwo_beam(n, r_in=rb - 0.05e-2, r_out=rb + 0.05e-2, z0=zs0, z1=zs1,
                                voltage=p["voltage"], seed=4000 + i)
    return dict(params=p, nodes=nodes, tris=tris, be=be, bt=bt, z_end=z_end, z=z, r=r, ur=ur,
                up=up, uz=uz, n=n)


def union(instances):
    """One mesh and one particle set holding all instances, shifted apart along z.

    Returns a dict with the union arrays and, per instance, the offsets of its nodes,
    triangles and particles (``node_off``, ``tri_off``, ``part_off``, each of length
    len(instances) + 1) and its z shift."""
    nodes, tris, be, bt, zs, rs, urs, ups, uzs = [], [], [], [], [], [], [], [], []
    node_off, tri_off, part_off, shift = [0], [0], [0], []
    z0 = 0.0
    for ins in instances:
        nn = ins["nodes"].copy()
        nn[:, 0] += z0
        nodes.append(nn)
        tris.append(ins["tris"] + node_off[-1])
        be.append(ins["be"] + node_off[-1])
        bt.append(ins["bt"])
        zs.append(ins["z"] + z0)
        rs.append(ins["r"])
        urs.append(ins["ur"])
        ups.append(ins["up"])
        uzs.append(ins["uz"])
        shift.append(z0)
        node_off.append(node_off[-1] + len(ins["nodes"]))
        tri_off.append(tri_off[-1] + len(ins["tris"]))
        part_off.append(part_off[-1] + len(ins["z"]))
        z0 += ins["z_end"] + GAP
    cat = np.concatenate
    return dict(nodes=cat(nodes), tris=cat(tris).astype(np.int32),
                be=cat(be).astype(np.int32), bt=cat(bt).astype(np.int32),
                z=cat(zs), r=cat(rs), ur=cat(urs), up=cat(ups), uz=cat(uzs),
                node_off=np.array(node_off), tri_off=np.array(tri_off),
                part_off=np.array(part_off), shift=np.array(shift))
