"""Seeded particle samplers.  Positions are physical (z, rho); momenta are u = gamma*v
in the local (rho, phi, z) frame of each particle."""
import numpy as np


def maxwellian(n, sigma_u, rng, drift=(0.0, 0.0, 0.0)):
    """Gaussian momenta u = gamma v with standard deviation sigma_u per component."""
    u = rng.normal(0.0, sigma_u, (n, 3)) + np.asarray(drift, float)[None, :]
    return u[:, 0].copy(), u[:, 1].copy(), u[:, 2].copy()


def uniform_in_volume_rect(n, z0, z1, r0, r1, rng):
    """Uniform in the volume of the annular cylinder r0<=rho<=r1, z0<=z<=z1.

    The volume element is rho drho dphi dz, so rho^2 is uniform."""
    z = rng.uniform(z0, z1, n)
    rho = np.sqrt(rng.uniform(r0 * r0, r1 * r1, n))
    return z, rho


def cavity_particles(n=10_000, a=0.5, L=1.0, sigma_u=0.01, seed=2000, margin=1e-3):
    """Electrons uniform in the cavity volume with a thermal spread sigma_u (c = 1)."""
    rng = np.random.default_rng(seed)
    z, rho = uniform_in_volume_rect(n, margin, L - margin, 0.0, a - margin, rng)
    ur, up, uz = maxwellian(n, sigma_u, rng)
    return z, rho, ur, up, uz


def bwo_beam(n, r_in=0.85e-2, r_out=0.95e-2, z0=3e-2, z1=3e-2 + 12 * 1.67e-2,
             voltage=400e3, thermal=1e-3, seed=2002, c=299792458.0,
             mc2_volts=510998.95):
    """Annular relativistic electron beam drifting along +z.

    gamma = 1 + V / (m c^2 / e); u_z = gamma beta c; momenta get a Gaussian thermal
    spread of ``thermal * u_z`` on all three components."""
    rng = np.random.default_rng(seed)
    gamma = 1.0 + voltage / mc2_volts
    beta = np.sqrt(1.0 - 1.0 / (gamma * gamma))
    uz0 = gamma * beta * c
    z, rho = uniform_in_volume_rect(n, z0, z1, r_in, r_out, rng)
    ur, up, uz = maxwellian(n, thermal * uz0, rng, drift=(0.0, 0.0, uz0))
    return z, rho, ur, up, uz


def uniform_in_mesh(nodes, tris, n, seed, sigma_u=0.0, drift=(0.0, 0.0, 0.0), shrink=1e-6):
    """Points uniform in area over the mesh (about n / N2 per triangle).

    ``shrink`` keeps samples a hair inside their triangle so that no sample lies on
    an edge.  Returns (z, rho, u_rho, u_phi, u_z)."""
    rng = np.random.default_rng(seed)
    p = nodes[tris]
    area = 0.5 * np.abs((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                        - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    t = rng.choice(len(tris), size=n, p=area / area.sum())
    r1 = rng.random(n)
    r2 = rng.random(n)
    s = np.sqrt(r1)
    b = np.stack([1.0 - s, s * (1.0 - r2), s * r2], 1)
    b = (1.0 - 3 * shrink) * b + shrink
    xy = np.einsum("nk,nkd->nd", b, p[t])
    ur, up, uz = maxwellian(n, sigma_u, rng, drift)
    return xy[:, 0].copy(), xy[:, 1].copy(), ur, up, uz
