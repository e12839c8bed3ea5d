"""Sources either side of the particle loop: the static gun field (Sec. 5.3, the cathode-
anode voltage by a Poisson solve), emission of particles from a cathode line (Secs. 5.2,
5.3), and the space-charge-limited current of a planar gap that a diode settles to.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Emission draws are counter-based so that the GPU library, which implements the same
published generator on its own, makes the same particles: for particle id p and draw j,
x = splitmix64(seed + 8 p + j) (Steele, Lea and Flood 2014, the finaliser Vigna uses
for seeding), u = (x >> 11 + 1/2) 2^-53 in (0, 1)."""
import math

import numpy as np
import scipy.sparse.linalg as spla
from scipy.integrate import quad

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """The splitmix64 output function of a uint64 array (arithmetic mod 2^64)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def uniforms(seed, pids, n_draws):
    """(len(pids), n_draws) uniforms in (0, 1) from the particle ids."""
    p = np.asarray(pids, np.uint64)[:, None]
    j = np.arange(n_draws, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        x = np.uint64(seed) + np.uint64(8) * p + j
    return ((splitmix64(x) >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53


def emitted(z0, rho0, rho1, u_normal, u_thermal, seed, pids):
    """Birth states of the particles with the given ids on the line z = z0, rho in
    [rho0, rho1]: uniform in area (density proportional to rho), momenta u = gamma v with
    independent normal components of spread u_thermal about (0, 0, u_normal)
    (Box-Muller on draws 1, 2 and 3, 4).  Returns z, rho, u_rho, u_phi, u_z."""
    u = uniforms(seed, pids, 5)
    rho = np.sqrt(rho0 * rho0 + u[:, 0] * (rho1 * rho1 - rho0 * rho0))
    r1 = np.sqrt(-2.0 * np.log(u[:, 1]))
    r3 = np.sqrt(-2.0 * np.log(u[:, 3]))
    ur = u_thermal * r1 * np.cos(2.0 * math.pi * u[:, 2])
    up = u_thermal * r1 * np.sin(2.0 * math.pi * u[:, 2])
    uz = u_normal + u_thermal * r3 * np.cos(2.0 * math.pi * u[:, 4])
    return np.full(len(rho), float(z0)), rho, ur, up, uz


def static_potential(mesh, star_eps, held_nodes, held_phi, charge=None):
    """Static field of the electrodes: the node potential phi with phi fixed at
    held_nodes and D_div star_eps D_div^T phi = Q at every other node (the discrete Gauss
    law D_div D = Q for D = star_eps E, E = -grad phi, whose Whitney-1 edge values are
    D_div^T phi: phi at the tail minus phi at the head), i.e. zero normal flux where no
    potential is held.  Q (node charges in the units of star_eps, per radian) defaults to
    zero.  Returns (phi, E_static)."""
    L = (mesh.Ddiv @ star_eps @ mesh.Ddiv.T).tocsr()
    held = np.zeros(mesh.N0, bool)
    held[np.asarray(held_nodes)] = True
    phi = np.zeros(mesh.N0)
    phi[np.asarray(held_nodes)] = held_phi
    free = ~held
    rhs = -(L[free][:, held] @ phi[held])
    if charge is not None:
        rhs = rhs + np.asarray(charge, float)[free]
    phi[free] = spla.spsolve(L[free][:, free].tocsc(), rhs)
    return phi, mesh.Ddiv.T @ phi


def child_langmuir_planar(V, d, q_over_m, eps0, c):
    """Space-charge-limited current density of a planar gap of width d at voltage V,
    relativistic, particles leaving the emitter at rest.  With the field zero at the
    emitter, the first integral of eps0 phi'' = J / v is (eps0/2) phi'^2 = J (c / qm)
    sqrt(gamma^2 - 1), gamma = 1 + qm phi / c^2, so d = int_0^V dphi / phi' gives
      J = eps0 qm / (2 c d^2) (int_0^V (gamma^2 - 1)^(-1/4) dphi)^2.
    The integral is taken with phi = V s^4 (smooth integrand)."""
    qm = abs(q_over_m)

    def f(s):
        if s == 0.0:
            return 0.0
        x = qm * V * s ** 4 / (c * c)          # gamma - 1
        return 4.0 * V * s ** 3 * (x * (2.0 + x)) ** -0.25

    integral, _ = quad(f, 0.0, 1.0, epsabs=0.0, epsrel=1e-13, limit=200)
    return eps0 * qm / (2.0 * c * d * d) * integral ** 2
