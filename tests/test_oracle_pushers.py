"""Pins of the oracle's two velocity updates of Eq. DLE (Sec. 3.3): each is checked
against the implicit equation it solves, and against closed forms in uniform fields.
CPU only.

Boris: u1 - u0 = 2h (E + (u0 + u1)/2 / gamma(u0 + h E) x B);
Vay:   u1 - u0 = 2h (E + (v0 + v1)/2 x B), v = u / gamma(u);  h = q dt / (2 m)."""
import math

import numpy as np
import pytest

from oracle import particles as P

C = 1.0


def _gamma(u):
    return np.sqrt(1.0 + np.sum(u * u, -1) / C ** 2)


def _random_case(n, seed, umax=3.0, emax=0.5, bmax=2.0):
    rng = np.random.default_rng(seed)
    u = rng.uniform(-umax, umax, (n, 3))
    E = rng.uniform(-emax, emax, (n, 3))
    B = rng.uniform(-bmax, bmax, (n, 3))
    return u, E, B


@pytest.mark.parametrize("h", [0.01, 0.2])
def test_boris_solves_the_momentum_mean_form(h):
    u0, E, B = _random_case(500, 1)
    u1 = P.kick(P.BORIS, u0, E, B, h, C)
    gm = _gamma(u0 + h * E)[:, None]
    rhs = 2 * h * (E + np.cross(0.5 * (u0 + u1) / gm, B))
    assert np.abs(u1 - u0 - rhs).max() < 1e-13 * np.abs(u0).max()


@pytest.mark.parametrize("h", [0.01, 0.2])
def test_vay_solves_the_velocity_mean_form(h):
    u0, E, B = _random_case(500, 2)
    u1 = P.kick(P.VAY, u0, E, B, h, C)
    vm = 0.5 * (u0 / _gamma(u0)[:, None] + u1 / _gamma(u1)[:, None])
    rhs = 2 * h * (E + np.cross(vm, B))
    assert np.abs(u1 - u0 - rhs).max() < 1e-13 * np.abs(u0).max()
    # and Boris does not satisfy the velocity-mean form (the pin tells them apart)
    ub = P.kick(P.BORIS, u0, E, B, h, C)
    vb = 0.5 * (u0 / _gamma(u0)[:, None] + ub / _gamma(ub)[:, None])
    assert np.abs(ub - u0 - 2 * h * (E + np.cross(vb, B))).max() > 1e-6


@pytest.mark.parametrize("pusher", [P.BORIS, P.VAY])
def test_pure_electric_field_is_a_full_kick(pusher):
    u0, E, _ = _random_case(200, 3)
    u1 = P.kick(pusher, u0, E, np.zeros(3), 0.1, C)
    assert np.abs(u1 - (u0 + 0.2 * E)).max() < 1e-15 * np.abs(u0).max() * 10


@pytest.mark.parametrize("pusher", [P.BORIS, P.VAY])
def test_pure_magnetic_field_rotates_by_the_closed_form_angle(pusher):
    """B along z: |u| and u_z are kept; (u_rho, u_phi) turns by 2 atan(h |B| / gamma)
    per step, clockwise for h B_z > 0 (d u/dt = (q/m) v x B in the right-handed
    (rho, phi, z) frame)."""
    rng = np.random.default_rng(4)
    u0 = rng.uniform(-3, 3, (100, 3))
    bz, h = 1.5, 0.07
    u1 = P.kick(pusher, u0, np.zeros(3), np.array([0.0, 0.0, bz]), h, C)
    assert np.allclose(np.linalg.norm(u1, axis=1), np.linalg.norm(u0, axis=1), rtol=1e-14)
    assert np.allclose(u1[:, 2], u0[:, 2], rtol=0, atol=1e-14)
    ang0 = np.arctan2(u0[:, 1], u0[:, 0])
    ang1 = np.arctan2(u1[:, 1], u1[:, 0])
    turn = np.angle(np.exp(1j * (ang0 - ang1)))
    expect = 2 * np.arctan(h * bz / _gamma(u0))
    assert np.allclose(turn, expect, rtol=0, atol=1e-13)


@pytest.mark.parametrize("gam", [1.01, 10.0, 1000.0])
def test_vay_leaves_a_force_free_particle_unaccelerated(gam):
    """E = -v x B (crossed fields, the particle at the drift velocity): Eq. DLE's solution
    is u1 = u0, which the Vay update returns to rounding; Boris does not at gamma = 1.01."""
    umag = math.sqrt(gam ** 2 - 1) * C
    u0 = np.array([[0.0, umag, 0.0]])
    B = np.array([0.0, 0.0, 2.0])
    E = -np.cross(u0[0] / gam, B)
    u1 = P.kick(P.VAY, u0, E, B, 0.05, C)
    assert np.abs(u1 - u0).max() <= 1e-14 * umag
    if gam < 2:
        ub = P.kick(P.BORIS, u0, E, B, 0.05, C)
        assert np.abs(ub - u0).max() > 1e-6 * umag


def test_cycle_uses_the_selected_pusher():
    """Through a whole particle step of the cycle: a particle moving in phi at the E x B
    drift speed (uniform E_rho = -v_phi B_z, guide field B_z) is force-free, so with the
    Vay update its momentum only turns with the rotation back to the meridian plane, by
    theta = atan2(v_phi dt, rho) (Eq. DNE); Boris leaves a visible error at gamma = 1.01."""
    import workloads as W
    from oracle import OracleSim

    nodes, tris, be, bt = W.rect_mesh(1.0, 1.0, 400, 21)
    out = {}
    for pusher in (P.BORIS, P.VAY):
        s = OracleSim(nodes, tris, be, bt)
        m = s.mesh
        dt, bz, gam = 0.5 * s.dt_max, 10.0, 1.01
        s.create(dt, bz=bz)
        s.pusher = pusher
        uphi = math.sqrt(gam ** 2 - 1.0)
        E_rho = -(uphi / gam) * bz
        d = m.nodes[m.edge_nodes[:, 1]] - m.nodes[m.edge_nodes[:, 0]]
        s.set_fields(E_rho * d[:, 1], np.zeros(m.N2))        # line integrals of E_rho
        rho0 = 0.5
        s.inject([0.5], [rho0], [0.0], [uphi], [0.0], 1.0, 1.0, 1e-9)
        s.push_particles(s.field_b_half())
        out[pusher] = s.u[0].copy()
    th = math.atan2(uphi / gam * dt, rho0)
    expect = np.array([math.sin(th) * uphi, math.cos(th) * uphi, 0.0])
    assert np.abs(out[P.VAY] - expect).max() <= 1e-14 * uphi
    assert np.abs(out[P.BORIS] - expect).max() > 1e-9 * uphi
