"""Initial field values: analytic cavity modes sampled as edge/face degrees of freedom,
and seeded random field values."""
import numpy as np
from scipy.special import jn_zeros, j0, j1

# 8-point Gauss-Legendre on [0, 1]
_gx, _gw = np.polynomial.legendre.leggauss(8)
_GX = 0.5 * (_gx + 1.0)
_GW = 0.5 * _gw


def tm0np_omega(a, L, n, p, c=1.0):
    """Angular frequency of the TM_0np mode of a closed cylinder (radius a, length L)."""
    k = jn_zeros(0, n)[-1] / a
    return c * np.sqrt(k * k + (p * np.pi / L) ** 2)


def _tm0np_E(z, rho, a, L, n, p):
    """Divergence-free TM_0np electric field pattern (E_z, E_rho).

    E_z = J0(k rho) cos(beta z), E_rho = (beta / k) J1(k rho) sin(beta z), with
    k = x_0n / a and beta = p pi / L: tangential E vanishes on rho = a and z = 0, L."""
    k = jn_zeros(0, n)[-1] / a
    beta = p * np.pi / L
    ez = j0(k * rho) * np.cos(beta * z)
    er = (beta / k) * j1(k * rho) * np.sin(beta * z)
    return ez, er


def tm0np_edge_dofs(nodes, edge_nodes, a=0.5, L=1.0, n=1, p=0, amp=1.0):
    """Line integrals of the mode's E along each edge, from edge_nodes[:,0] to [:,1]."""
    pa = nodes[edge_nodes[:, 0]]
    pb = nodes[edge_nodes[:, 1]]
    d = pb - pa
    out = np.zeros(len(edge_nodes))
    for x, w in zip(_GX, _GW):
        q = pa + x * d
        ez, er = _tm0np_E(q[:, 0], q[:, 1], a, L, n, p)
        out += w * (ez * d[:, 0] + er * d[:, 1])
    return amp * out


def random_edge_values(n, scale, seed):
    """Seeded uniform values in [-scale, scale]."""
    return np.random.default_rng(seed).uniform(-scale, scale, n)
