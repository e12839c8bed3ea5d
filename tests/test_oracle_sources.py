"""Pins of the oracle's sources (oracle/sources.py): the counter-based generator against
its published outputs, the emitted distributions, the static-field Laplace problem
against exact and closed-form solutions, the planar space-charge-limited current against
its classical and ultra-relativistic limits and against the ODE it comes from, and charge
conservation with particles born every step.  CPU only."""
import math

import numpy as np
import pytest
from scipy import stats
from scipy.integrate import solve_ivp

import workloads as W
from oracle import OracleSim, sources as S
from oracle.operators import Mesh, hodge_eps

EPS0, QM, C = 8.8541878128e-12, 1.75882001076e11, 299792458.0


def test_splitmix64_published_outputs():
    """The first outputs of the generator from state 0 (Vigna's reference splitmix64.c):
    state x gives splitmix64(x), and the state advances by the golden gamma."""
    gamma = 0x9E3779B97F4A7C15
    states = np.array([0, gamma, (2 * gamma) % 2 ** 64], np.uint64)
    out = S.splitmix64(states)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                     0x06C45D188009454F]


def test_uniform_draws_are_uniform_and_distinct():
    u = S.uniforms(12345, np.arange(20000), 5)
    assert u.min() > 0 and u.max() < 1
    for j in range(5):
        assert stats.kstest(u[:, j], "uniform").pvalue > 1e-3
    assert len(np.unique(u)) == u.size
    # counter-based: a particle's draws do not depend on which others are drawn
    assert np.array_equal(S.uniforms(12345, np.array([777]), 5)[0], u[777])


def test_emitted_distributions():
    z, r, ur, up, uz = S.emitted(0.3, 0.2, 0.5, 2.0, 0.1, 99, np.arange(40000))
    assert np.all(z == 0.3) and r.min() >= 0.2 and r.max() <= 0.5
    # uniform in area: F(rho) = (rho^2 - rho0^2) / (rho1^2 - rho0^2)
    cdf = lambda x: (np.clip(x, 0.2, 0.5) ** 2 - 0.04) / (0.25 - 0.04)
    assert stats.kstest(r, cdf).pvalue > 1e-3
    for comp, mean in ((ur, 0.0), (up, 0.0), (uz, 2.0)):
        assert stats.kstest((comp - mean) / 0.1, "norm").pvalue > 1e-3


def test_static_potential_of_a_planar_gap_is_exact():
    """phi held at 0 on z = 0 and V on z = L, free elsewhere (the axis and the outer wall
    then carry zero normal flux): the exact solution V z / L lies in the Whitney-0 space,
    so the discrete one equals it, and each edge value is the line integral of the
    uniform field, -V (z_head - z_tail) / L."""
    nodes, tris, be, bt = W.cavity_mesh(a=0.5, L=1.0, n_tri=1500, seed=5)
    m = Mesh(nodes, tris, be, bt)
    V = 3.0
    held = np.flatnonzero((m.nodes[:, 0] == 0.0) | (m.nodes[:, 0] == 1.0))
    phi, E = S.static_potential(m, hodge_eps(m), held, V * m.nodes[held, 0])
    assert np.abs(phi - V * m.nodes[:, 0]).max() < 1e-12 * V
    dz = m.nodes[m.edge_nodes[:, 1], 0] - m.nodes[m.edge_nodes[:, 0], 0]
    assert np.abs(E + V * dz).max() < 1e-12 * V


def test_static_potential_converges_to_an_axisymmetric_harmonic():
    """phi = rho^2 - 2 z^2 is harmonic in 3D cylindrical coordinates and has zero radial
    derivative on the axis; held at the walls, the discrete solution's nodal error is
    second order in the mesh size."""
    errs = []
    for n in (800, 3200):
        nodes, tris, be, bt = W.cavity_mesh(a=0.5, L=1.0, n_tri=n, seed=6)
        m = Mesh(nodes, tris, be, bt)
        exact = m.nodes[:, 1] ** 2 - 2.0 * (m.nodes[:, 0] - 0.5) ** 2
        held = np.flatnonzero(m.node_on_pec)
        phi, _ = S.static_potential(m, hodge_eps(m), held, exact[held])
        errs.append(np.abs(phi - exact).max())
    assert errs[0] < 2e-2
    assert errs[1] < errs[0] / 2.5      # h halves: about 4x


def test_child_langmuir_limits():
    d = 0.01
    for V in (1e-3, 1.0):
        J = S.child_langmuir_planar(V, d, QM, EPS0, C)
        classical = 4.0 * EPS0 / 9.0 * math.sqrt(2.0 * QM) * V ** 1.5 / d ** 2
        assert abs(J / classical - 1.0) < 5e-7
    rel = [S.child_langmuir_planar(V, d, QM, EPS0, C) / (2.0 * EPS0 * C * V / d ** 2) - 1
           for V in (1e10, 1e12)]
    assert abs(rel[1]) < 2e-3 and abs(rel[1]) < abs(rel[0]) / 5


@pytest.mark.parametrize("V", [1e4, 1e5, 1e6])
def test_child_langmuir_current_closes_the_gap(V):
    """Integrate eps0 phi'' = J / v(phi) from the emitter with phi = phi' = 0 at the
    computed J: the potential reaches V exactly at x = d."""
    d = 0.01
    J = S.child_langmuir_planar(V, d, QM, EPS0, C)

    def v(phi):
        g = 1.0 + QM * phi / C ** 2
        return C * math.sqrt(1.0 - 1.0 / (g * g))

    # start off the singular point with the classical small-x series
    x0 = 1e-7 * d
    k = (9.0 * J / (4.0 * EPS0 * math.sqrt(2.0 * QM))) ** (2.0 / 3.0)
    y0 = [k * x0 ** (4.0 / 3.0), 4.0 / 3.0 * k * x0 ** (1.0 / 3.0)]
    sol = solve_ivp(lambda x, y: [y[1], J / (EPS0 * v(y[0]))], (x0, d), y0, rtol=1e-10,
                    atol=1e-12 * V)
    assert abs(sol.y[0, -1] / V - 1.0) < 1e-4


def test_charge_conservation_with_particles_born_every_step():
    """200 particles emitted at the start of each of 20 steps into a random field: the DCE
    residual stays at round-off, and the Gauss-law residual with the born charge taken
    out stays constant."""
    nodes, tris, be, bt = W.cavity_mesh(a=0.5, L=1.0, n_tri=800, seed=7)
    s = OracleSim(nodes, tris, be, bt)
    s.create(0.5 * s.dt_max, bz=0.2)
    m = s.mesh
    s.set_fields(W.random_edge_values(m.N1, 0.05, 1), np.zeros(m.N2))
    s.set_emitter(0.02, 0.0, 0.3, 200, 1.0, 0.2, 5, -1.0, 1.0, 1e-3)
    res0 = None
    for k in range(20):
        s.step()
        r = s.dce_residual()
        assert np.abs(r).max() * s.dt < 1e-12 * max(np.abs(s.Q).max(), 1e-30)
        g = s.dgl_residual()
        if res0 is None:
            res0 = g.copy()
        assert np.abs(g - res0).max() < 1e-10 * np.abs(s.Q_born).max()
    assert len(s.tri) == 20 * 200 and s.counters[2] > 0


def test_gauss_law_of_a_charged_shell_fixes_the_ring_normalisation():
    """Macro-particles on a cylindrical shell rho = 0.4 inside a grounded tube rho = 1
    (ends without normal flux: an infinitely long line).  Their Eq. charge deposit (q_src =
    w q / (2 pi) per radian) drives the discrete Gauss law through star_eps (also per
    radian); outside the shell the potential must fall as Q_tot / (2 pi eps0 L) ln(rho),
    Q_tot the 3D charge N w q.  A missing or doubled 2 pi shows as a factor 6.28."""
    from oracle import particles as P
    nodes, tris, be, bt = W.cavity_mesh(a=1.0, L=4.0, n_tri=6000, seed=12)
    s = OracleSim(nodes, tris, be, bt)
    m = s.mesh
    n, w, q = 20000, 2e-3, -1.0
    z = (np.arange(n) + 0.5) * (4.0 / n)     # evenly spread: no shot noise in the line charge
    r = np.full(n, 0.4)
    tri, lam = P.locate(m, z, r)
    Q = np.zeros(m.N0)
    P.deposit_charge(s.pm, tri, np.ascontiguousarray(lam), w * q / (2 * math.pi), Q)
    held = np.flatnonzero(np.isclose(m.nodes[:, 1], 1.0))
    phi, _ = S.static_potential(m, s.star_eps, held, np.zeros(len(held)), charge=Q)
    k = np.flatnonzero((m.nodes[:, 1] > 0.55) & (m.nodes[:, 1] < 0.95)
                       & (m.nodes[:, 0] > 1.0) & (m.nodes[:, 0] < 3.0))
    expect = n * w * q / (2 * math.pi * 1.0 * 4.0) * np.log(1.0 / m.nodes[k, 1])
    assert np.abs(phi[k] - expect).max() < 0.005 * np.abs(expect).max()


def test_static_field_drives_particles_but_not_the_leapfrog():
    """The gun field of a planar gap (phi = V z / L, edge values -V dz / L) is added to E
    at the gather only: particles at rest gain u_z = (q/m)(-V/L) dt in one step, while
    the dynamic fields, with no current (weight 0), stay exactly zero."""
    nodes, tris, be, bt = W.cavity_mesh(a=0.5, L=1.0, n_tri=800, seed=5)
    s = OracleSim(nodes, tris, be, bt)
    m = s.mesh
    dt = 0.5 * s.dt_max
    s.create(dt)
    V = 2.0
    held = np.flatnonzero((m.nodes[:, 0] == 0.0) | (m.nodes[:, 0] == 1.0))
    _, Es = S.static_potential(m, s.star_eps, held, V * m.nodes[held, 0])
    s.set_static_field(Es)
    rng = np.random.default_rng(3)
    n = 40
    z, r = rng.uniform(0.2, 0.8, n), rng.uniform(0.1, 0.4, n)
    q, mass = -1.0, 2.0
    s.inject(z, r, np.zeros(n), np.zeros(n), np.zeros(n), q, mass, 0.0)
    s.step()
    assert np.allclose(s.u[:, 2], q / mass * (-V) * dt, rtol=1e-12, atol=0)
    assert np.abs(s.u[:, :2]).max() < 1e-12 * V * dt
    assert np.all(s.E == 0) and np.all(s.B == 0)


def _unmix(y):
    """Inverse of the splitmix64 output function (each xor-shift and odd multiplier is a
    bijection of 64-bit words), so that a state with a chosen output can be built."""
    M = 2 ** 64

    def unshift(v, s):
        x = v
        for _ in range(64 // s + 1):
            x = v ^ (x >> s)
        return x

    z = unshift(y, 31)
    z = (z * pow(0x94D049BB133111EB, -1, M)) % M
    z = unshift(z, 27)
    z = (z * pow(0xBF58476D1CE4E5B9, -1, M)) % M
    z = unshift(z, 30)
    return (z - 0x9E3779B97F4A7C15) % M


def test_uniform_draws_stay_inside_the_open_interval_at_the_extremes():
    """The generator's smallest and largest outputs (0 and 2^64 - 1, reached from states
    built by inverting it) map to 2^-54 and 1 - 2^-54: the draws never reach 0, whose
    logarithm the Box-Muller step takes, nor 1."""
    for out, u in ((0, 2.0 ** -54), (2 ** 64 - 1, 1.0 - 2.0 ** -54)):
        x = _unmix(out)
        assert int(S.splitmix64(np.array([x], np.uint64))[0]) == out
        assert S.uniforms(x, np.array([0]), 1)[0, 0] == u


def test_emitted_transverse_momenta_are_independent_normals():
    """Box-Muller pairs: u_rho and u_phi are independent, so (u_rho^2 + u_phi^2) / (2 s^2)
    follows the unit exponential law and their correlation vanishes."""
    sig = 0.1
    _, _, ur, up, _ = S.emitted(0.3, 0.2, 0.5, 2.0, sig, 7, np.arange(40000))
    assert stats.kstest((ur ** 2 + up ** 2) / (2 * sig ** 2), "expon").pvalue > 1e-3
    assert abs(np.corrcoef(ur, up)[0, 1]) < 0.03


def test_successive_emissions_continue_the_particle_ids():
    """Each step's births are new particles: their ids continue the count, so two steps
    emit different draws, each the draws of its own ids."""
    nodes, tris, be, bt = W.cavity_mesh(a=0.5, L=1.0, n_tri=400, seed=7)
    s = OracleSim(nodes, tris, be, bt)
    s.create(0.5 * s.dt_max)
    s.set_emitter(0.02, 0.0, 0.3, 50, 1.0, 0.2, 5, -1.0, 1.0, 1e-3)
    s.emit()
    s.emit()
    for k in (0, 1):
        _, r, ur, up, uz = S.emitted(0.02, 0.0, 0.3, 1.0, 0.2, 5, np.arange(50 * k, 50 * k + 50))
        assert np.array_equal(s.u[50 * k:50 * k + 50], np.stack([ur, up, uz], 1))
    assert not np.any(np.isin(s.u[:50, 0], s.u[50:, 0]))
