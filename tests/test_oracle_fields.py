"""Pins of the oracle's field solver: cavity resonances against the Bessel-zero closed
form (Sec. 4.1, Table 1) and the stability limit of the leapfrog scheme.  CPU only."""
import math

import numpy as np
import pytest
from scipy.optimize import least_squares

import workloads as W
from oracle import OracleSim


@pytest.fixture(scope="module")
def cavity():
    """The 0.5 x 1 normalised cavity (c = 1) with about 2000 triangles."""
    return OracleSim(*W.cavity_mesh())


def _two_tone_fit(t, a, w0, w1):
    def res(p):
        return (p[0] * np.cos(p[2] * t) + p[1] * np.sin(p[2] * t)
                + p[3] * np.cos(p[5] * t) + p[4] * np.sin(p[5] * t) - a)
    r = least_squares(res, [a[0], 0.0, w0, 0.0, 0.0, w1], x_scale="jac")
    return r.x


def test_cavity_tm010_tm011_frequencies(cavity):
    """E^0 = TM010 + TM011 line integrals, B^{-1/2} = 0, 1000 steps at half the stable
    step; the projections on the two mode patterns oscillate at the closed-form
    frequencies omega = c sqrt((x_0n/a)^2 + (p pi/L)^2) within 0.5%."""
    s = cavity
    m = s.mesh
    dt = 0.5 * s.dt_max
    s.create(dt)
    P0 = W.tm0np_edge_dofs(m.nodes, m.edge_nodes, 0.5, 1.0, 1, 0)
    P1 = W.tm0np_edge_dofs(m.nodes, m.edge_nodes, 0.5, 1.0, 1, 1)
    s.set_fields(P0 + P1, np.zeros(m.N2))
    a0, a1 = [], []
    for _ in range(1000):
        a0.append(s.E @ P0)
        a1.append(s.E @ P1)
        s.step()
    t = np.arange(1000) * dt
    w010 = W.tm0np_omega(0.5, 1.0, 1, 0)
    w011 = W.tm0np_omega(0.5, 1.0, 1, 1)
    p0 = _two_tone_fit(t, np.array(a0), w010, w011)
    p1 = _two_tone_fit(t, np.array(a1), w011, w010)
    # the dominant tone of each projection
    f0 = p0[2] if np.hypot(p0[0], p0[1]) > np.hypot(p0[3], p0[4]) else p0[5]
    f1 = p1[2] if np.hypot(p1[0], p1[1]) > np.hypot(p1[3], p1[4]) else p1[5]
    assert abs(f0 - w010) / w010 < 5e-3
    assert abs(f1 - w011) / w011 < 5e-3


def test_stability_limit(cavity):
    """At half the estimated limit the field energy stays bounded; 5% above it the
    leapfrog diverges."""
    m = cavity.mesh
    E0 = W.random_edge_values(m.N1, 1.0, 3)

    def run(f, n):
        s = OracleSim.__new__(OracleSim)
        s.__dict__.update(cavity.__dict__)
        s.dt = f * cavity.dt_max
        s.set_fields(E0, np.zeros(m.N2))
        s.J = np.zeros(m.N1)
        e0 = s.field_energy()
        emax = e0
        for _ in range(n):
            Bh = s.field_b_half()
            s.field_e(Bh)
            s.B = Bh
            emax = max(emax, s.field_energy())
            if emax > 1e8 * e0:
                break
        return emax / e0

    assert run(0.5, 1000) < 2.0
    assert run(1.05, 400) > 1e6


def test_field_energy_of_uniform_fields_closed_form():
    """The energy densities eps0 E^2 / 2 and B^2 / (2 mu0) integrated per radian
    (int rho dz drho = a^2 L / 2 over the cavity): a uniform E (exact in Whitney 1-forms)
    and a uniform B_phi (B_f = B0 A_f) must give eps0 E0^2 a^2 L / 4 and
    B0^2 a^2 L / (4 mu0), for any eps0 and mu0."""
    from oracle.operators import Mesh, hodge_eps, hodge_mu_inv, field_energy
    a, L = 0.5, 1.0
    m = Mesh(*W.cavity_mesh(a=a, L=L, n_tri=600, seed=4))
    eps0, mu0 = 2.5, 0.6
    se, mi = hodge_eps(m, eps0), hodge_mu_inv(m, mu0)
    d = m.nodes[m.edge_nodes[:, 1]] - m.nodes[m.edge_nodes[:, 0]]
    E0, B0 = 0.7, 1.3
    for comp in (0, 1):
        We = field_energy(m, se, mi, E0 * d[:, comp], np.zeros(m.N2))
        assert abs(We - eps0 * E0 ** 2 * a * a * L / 4) < 1e-12 * We
    Wm = field_energy(m, se, mi, np.zeros(m.N1), B0 * m.area)
    assert abs(Wm - B0 ** 2 * a * a * L / (4 * mu0)) < 1e-12 * Wm


def test_conducting_walls_short_the_tangential_field():
    """A uniform E_z set in a closed conducting cavity: the walls hold no tangential E
    (on their edges E = 0, at every step), so the field is not curl-free next to them.
    Its circulation then lives only on faces that touch a wall (every face along the tube
    wall, whose edges run along z), and the first B half step is zero everywhere else;
    the field oscillates instead of staying put."""
    from oracle.operators import BC_PEC
    s = OracleSim(*W.cavity_mesh(n_tri=800, seed=11))
    m = s.mesh
    s.create(0.5 * s.dt_max)
    d = m.nodes[m.edge_nodes[:, 1]] - m.nodes[m.edge_nodes[:, 0]]
    E0 = 0.3
    s.set_fields(E0 * d[:, 0], np.zeros(m.N2))
    wall = m.edge_tag == BC_PEC
    touches = np.any(wall[m.tri_edges], axis=1)
    shorted = np.any((wall & (np.abs(d[:, 0]) > 0))[m.tri_edges], axis=1)   # the tube wall
    Bh = s.field_b_half()
    assert np.abs(Bh[~touches]).max() < 1e-14 * E0
    assert np.abs(Bh[shorted]).min() > 0.0
    for _ in range(50):
        s.step()
        assert np.all(s.E[wall] == 0.0)
    assert np.abs(s.B).max() > 1e-3 * E0
