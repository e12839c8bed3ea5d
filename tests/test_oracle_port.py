"""Pins of the oracle's output-port power (Secs. 5.1, 5.1.1: the Poynting flux through the
output plane) by closed forms.  CPU only."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import port as OP
from oracle.operators import Mesh


@pytest.fixture(scope="module")
def guide():
    """A straight guide, radius 0.5, length 1 (the plane z0 avoids the lattice rows)."""
    return Mesh(*W.rect_mesh(1.0, 0.5, 1200, 17))


def _uniform(mesh, e0, b0):
    """Edge values of a uniform E_rho = e0 (line integrals) and face values of a uniform
    B_phi = b0 (B_f = b0 A_f)."""
    d = mesh.nodes[mesh.edge_nodes[:, 1]] - mesh.nodes[mesh.edge_nodes[:, 0]]
    return e0 * d[:, 1], b0 * mesh.area


@pytest.mark.parametrize("rho0,rho1", [(0.0, 0.5), (0.1, 0.37)])
def test_uniform_fields_give_the_closed_form(guide, rho0, rho1):
    """E_rho = e0, B_phi = b0 everywhere: P = (2 pi / mu0) e0 b0 (rho1^2 - rho0^2) / 2."""
    E, B = _uniform(guide, 0.7, -1.3)
    mu0 = 1.7
    P = OP.port_power(guide, E, B, 0.4321, rho0, rho1, mu0)
    exact = math.pi / mu0 * 0.7 * -1.3 * (rho1 ** 2 - rho0 ** 2)
    assert abs(P - exact) <= 1e-12 * abs(exact)


def test_power_is_bilinear_and_follows_the_orientation(guide):
    """Reversing B reverses P; P is linear in E and in B; a field with E_rho = 0 (a uniform
    E_z) carries none."""
    rng = np.random.default_rng(3)
    E = rng.uniform(-1, 1, guide.N1)
    B = rng.uniform(-1, 1, guide.N2)
    P = OP.port_power(guide, E, B, 0.61, 0.0, 0.5)
    assert abs(OP.port_power(guide, E, -B, 0.61, 0.0, 0.5) + P) <= 1e-12 * abs(P)
    assert abs(OP.port_power(guide, 2 * E, 3 * B, 0.61, 0.0, 0.5) - 6 * P) <= 1e-12 * abs(P)
    d = guide.nodes[guide.edge_nodes[:, 1]] - guide.nodes[guide.edge_nodes[:, 0]]
    Ez = 0.9 * d[:, 0]
    assert abs(OP.port_power(guide, Ez, B, 0.61, 0.0, 0.5)) <= 1e-12 * np.abs(B).max()


def test_linear_in_z_field_gives_its_value_at_the_plane(guide):
    """E = (-c rho, a + c z) (in the Whitney 1-form space, whose fields are
    (alpha_z - beta rho, alpha_rho + beta z)) with uniform B_phi = b0: P is the closed form
    with E_rho = a + c z0 (pins the barycentric evaluation along z)."""
    a, c, b0, z0 = 0.3, 1.1, 0.8, 0.2718
    p0 = guide.nodes[guide.edge_nodes[:, 0]]
    p1 = guide.nodes[guide.edge_nodes[:, 1]]
    mid = 0.5 * (p0 + p1)
    d = p1 - p0
    # line integral of (-c rho, a + c z) along each straight edge
    E = -c * mid[:, 1] * d[:, 0] + (a + c * mid[:, 0]) * d[:, 1]
    B = b0 * guide.area
    P = OP.port_power(guide, E, B, z0, 0.0, 0.5)
    exact = math.pi * (a + c * z0) * b0 * 0.25
    assert abs(P - exact) <= 1e-12 * abs(exact)
