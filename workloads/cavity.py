"""The normalised cavity workload (c = eps0 = mu0 = 1): closed conducting cylinder of radius
a = 0.5 and length L = 1 in the meridian plane, a seeded jittered Delaunay mesh of about
2000 triangles (seed 1000), E^0 = line integrals of the TM010 + TM011 mode patterns,
B^{-1/2} = 0, and 10,000 electrons (q = -1, m = 1) uniform in volume with Maxwellian
momenta of spread 0.01 c (seed 2000), the macro-particle weight set so that the plasma
frequency is 0.01 of the TM010 frequency."""
import math

from .meshes import cavity_mesh
from .particles import cavity_particles
from .fields import tm0np_edge_dofs, tm0np_omega

CAVITY_A, CAVITY_L = 0.5, 1.0


def cavity_weight(n, a=CAVITY_A, L=CAVITY_L, wp_over_w010=0.01):
    """Weight w of n electron macro-particles in the cylinder volume V = pi a^2 L with
    omega_p^2 = (n w / V) q^2 / (eps0 m) = (wp_over_w010 omega_010)^2 (normalised units)."""
    wp = wp_over_w010 * tm0np_omega(a, L, 1, 0)
    return wp * wp * math.pi * a * a * L / n


def cavity_workload(n_particles=10_000, n_tri=2000, mesh_seed=1000, seed=2000, amp=1.0):
    nodes, tris, be, bt = cavity_mesh(CAVITY_A, CAVITY_L, n_tri, mesh_seed)
    z, r, ur, up, uz = cavity_particles(n_particles, CAVITY_A, CAVITY_L, 0.01, seed)
    return dict(nodes=nodes, tris=tris, be=be, bt=bt, z=z, r=r, ur=ur, up=up, uz=uz,
                q=-1.0, m=1.0, weight=cavity_weight(n_particles), amp=amp,
                w010=tm0np_omega(CAVITY_A, CAVITY_L, 1, 0),
                w011=tm0np_omega(CAVITY_A, CAVITY_L, 1, 1))


def cavity_modes(nodes, edge_nodes):
    """The TM010 and TM011 edge patterns (line integrals along each edge)."""
    return (tm0np_edge_dofs(nodes, edge_nodes, CAVITY_A, CAVITY_L, 1, 0),
            tm0np_edge_dofs(nodes, edge_nodes, CAVITY_A, CAVITY_L, 1, 1))
