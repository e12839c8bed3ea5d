"""Absorbing port layers (pic_sim_set_loss): graded conductivity profiles.

The paper ends its output ports and left walls with a PML (Sec. 5.3) without giving its
equations; a graded, impedance-matched lossy layer stands in for it.  The conductivity
rises as ((z - z_start) / (z_end - z_start))^order through the layer (z_end < z_start for
a layer on the left), evaluated at edge midpoints and face centroids, with the magnetic
conductivity sigma_m = sigma_e mu0 / eps0 (matched: a plane wave entering at normal
incidence sees no impedance step).  sigma_max from the usual grading rule for a target
normal-incidence reflection R: (order + 1) ln(1/R) eps0 c / (2 thickness)."""
import math

import numpy as np


def sigma_max_for(reflection, thickness, order=3, eps0=1.0, c=1.0):
    return (order + 1) * math.log(1.0 / reflection) * eps0 * c / (2.0 * thickness)


def graded_layer(nodes, edge_nodes, tris, z_start, z_end, sigma_max, order=3, eps0=1.0,
                 mu0=1.0):
    """(sigma_e per edge, sigma_m per face) of one layer; zero outside it."""
    nodes = np.asarray(nodes, float)

    def profile(z):
        x = (z - z_start) / (z_end - z_start)
        return np.where(x > 0.0, sigma_max * np.clip(x, 0.0, 1.0) ** order, 0.0)

    ze = 0.5 * (nodes[edge_nodes[:, 0], 0] + nodes[edge_nodes[:, 1], 0])
    zf = nodes[np.asarray(tris)][:, :, 0].mean(1)
    se = profile(ze)
    return se, profile(zf) * mu0 / eps0
