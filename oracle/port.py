"""Output-port power of the discrete fields: the Poynting flux through a plane z = z0
between rho0 and rho1 (the BWO's output signal, Secs. 5.1 and 5.1.1).  Test
infrastructure: plain, slow, FP64; shares no code with the library.

  P = (2 pi / mu0) int_rho0^rho1 E_rho(z0, rho) B_phi(z0, rho) rho drho

E is the Whitney 1-form field sum_e E_e (lam_a grad lam_b - lam_b grad lam_a) (edge e from
its tail a, the lower global node index, to its head b); B_phi is the Whitney 2-form value
B_f / A_f of the triangle, for a face array B given as B_f (pass the time-centred
(B^{n+1/2} + B^{n-1/2}) / 2 to get the value the gather of step n sees).
"""
import math

import numpy as np


def _barycentric(p, z, rho):
    A = np.array([[1.0, 1.0, 1.0], p[:, 0], p[:, 1]])
    return np.linalg.solve(A, np.array([1.0, z, rho]))


def e_rho(mesh, E, t, lam):
    """rho component of the Whitney 1-form field of edge values E in triangle t at the
    barycentric point lam."""
    g = mesh.grad[t]                       # (3, 2): d lam_k / dz, d lam_k / drho
    n3 = mesh.tris[t]
    out = 0.0
    for k in range(3):                     # local edge k joins local nodes k+1 and k+2
        i, j = (k + 1) % 3, (k + 2) % 3
        a, b = (i, j) if n3[i] < n3[j] else (j, i)
        out += E[mesh.tri_edges[t, k]] * (lam[a] * g[b, 1] - lam[b] * g[a, 1])
    return out


def port_power(mesh, E, B, z0, rho0, rho1, mu0=1.0):
    """P through z = z0, rho0 <= rho <= rho1: Simpson's rule on each triangle's chord (the
    integrand is quadratic along it, so the rule is exact)."""
    total = 0.0
    for t in range(mesh.N2):
        p = mesh.nodes[mesh.tris[t]]
        z = p[:, 0]
        if z.min() >= z0 or z.max() <= z0:
            continue
        cuts = []
        for i in range(3):
            j = (i + 1) % 3
            if (z[i] - z0) * (z[j] - z0) < 0.0:
                s = (z0 - z[i]) / (z[j] - z[i])
                cuts.append(p[i, 1] + s * (p[j, 1] - p[i, 1]))
        if len(cuts) != 2:
            raise ValueError("the plane passes through a node of triangle %d" % t)
        a, b = max(min(cuts), rho0), min(max(cuts), rho1)
        if b <= a:
            continue
        bphi = B[t] / mesh.area[t]
        f = [e_rho(mesh, E, t, _barycentric(p, z0, r)) * r for r in (a, 0.5 * (a + b), b)]
        total += (b - a) / 6.0 * (f[0] + 4.0 * f[1] + f[2]) * bphi
    return 2.0 * math.pi / mu0 * total
