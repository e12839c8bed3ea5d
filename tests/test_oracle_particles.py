"""Pins of the oracle's particle step (gather, Boris, move, walk, scatter) against closed
forms and exact identities.  CPU only."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import OracleSim
from oracle.operators import Mesh
from oracle import particles as TPart


def _grad_by_solve(p):
    A = np.array([[1.0, 1.0, 1.0], p[:, 0], p[:, 1]])
    return np.linalg.inv(A)[:, 1:]


def _lam_by_solve(p, z, r):
    A = np.array([[1.0, 1.0, 1.0], p[:, 0], p[:, 1]])
    return np.linalg.solve(A, np.array([1.0, z, r]))


@pytest.fixture(scope="module")
def cavity():
    nodes, tris, be, bt = W.cavity_mesh(n_tri=800, seed=11)
    return OracleSim(nodes, tris, be, bt)


def _fresh(sim):
    """A copy of a prepared simulation without particles and with zero fields."""
    s = OracleSim.__new__(OracleSim)
    s.__dict__.update({k: v for k, v in sim.__dict__.items()})
    m = s.mesh
    s.E, s.B, s.D = np.zeros(m.N1), np.zeros(m.N2), np.zeros(m.N1)
    s.Q, s.Q_prev, s.J, s.Qabs = np.zeros(m.N0), np.zeros(m.N0), np.zeros(m.N1), np.zeros(m.N0)
    s.tri, s.lam, s.u = np.zeros(0, np.int32), np.zeros((0, 3)), np.zeros((0, 3))
    s.q_src = 0.0
    s.counters = np.zeros(3, np.int64)
    return s


def test_current_is_line_integral_of_whitney_form(cavity):
    """Eq. current: J_e = (q/dt) int_{r^n}^{r^{n+1}} W1_e . dr.  A force-free particle
    with u_phi = 0 moves on a straight segment; inside one triangle the deposited
    current must equal the Gauss-quadrature line integral of W1 along it."""
    s = _fresh(cavity)
    m = s.mesh
    dt = 0.4 * s.dt_max
    s.create(dt)
    rng = np.random.default_rng(0)
    done = 0
    for t in rng.permutation(m.N2):
        p = m.nodes[m.tris[t]]
        lam0 = np.array([0.4, 0.35, 0.25])
        step = np.array([-0.2, -0.05, 0.25])
        r0 = lam0 @ p
        if r0[1] < 0.05:
            continue
        # scale the in-triangle displacement to half the distance light covers in dt
        f = 0.5 * s.c * dt / np.linalg.norm(step @ p)
        lam1 = lam0 + min(f, 1.0) * step
        d = lam1 @ p - r0
        s2 = _fresh(cavity)
        s2.create(dt)
        # u = gamma v with v = d/dt, u_phi = 0
        v = d / dt
        gam = 1.0 / math.sqrt(1.0 - (v @ v) / s2.c ** 2)
        q, mass, w = -1.0, 1.0, 1e-3
        s2.inject([r0[0]], [r0[1]], [gam * v[1]], [0.0], [gam * v[0]], q, mass, w)
        s2.step()
        G = _grad_by_solve(p)
        x, wq = np.polynomial.legendre.leggauss(3)
        x, wq = 0.5 * (x + 1), 0.5 * wq
        for k in range(3):
            a, b = m.edge_tail_head(t, k)
            val = sum(wi * ((l := lam0 + xi * (lam1 - lam0))[a] * G[b] - l[b] * G[a]) @ d
                      for xi, wi in zip(x, wq))
            ref = s2.q_src / dt * val
            assert abs(s2.J[m.tri_edges[t, k]] - ref) <= 1e-12 * abs(s2.q_src / dt)
        # no other edge receives current
        others = np.setdiff1d(np.arange(m.N1), m.tri_edges[t])
        assert np.all(s2.J[others] == 0)
        done += 1
        if done == 5:
            break


def _random_run(cavity, n, speed, steps, seed, bz=0.3):
    s = _fresh(cavity)
    m = s.mesh
    s.create(0.5 * s.dt_max, bz=bz)
    rng = np.random.default_rng(seed)
    s.set_fields(W.random_edge_values(m.N1, 0.05, seed), W.random_edge_values(m.N2, 1e-4, seed + 1))
    z, r, ur, up, uz = W.uniform_in_mesh(m.nodes, m.tris, n, seed, sigma_u=speed)
    s.inject(z, r, ur, up, uz, -1.0, 1.0, 1e-3)
    return s


def test_dce_exact_with_multi_cell_crossings(cavity):
    """Eq. DCE holds per step to round-off even when particles cross several cells."""
    s = _random_run(cavity, 3000, speed=3.0, steps=3, seed=3)
    # a step far above the field's stability limit: only the particle part is run
    s.dt = 12 * s.dt_max
    for _ in range(3):
        Qn = s.push_particles(s.field_b_half())
        s.Q_prev, s.Q = s.Q, Qn
        res = s.dce_residual()
        assert np.abs(res).max() * s.dt <= 1e-13 * abs(s.q_src) * 10
    assert s.counters[2] > 3 * 3000          # several crossings per particle per step
    assert s.counters[0] > 0                   # some absorbed at the walls


def test_dgl_residual_constant(cavity):
    """Eq. DGL_RSD_REL: D_div D^n - Q^n does not change from step to step."""
    s = _random_run(cavity, 2000, speed=0.5, steps=5, seed=4)
    r0 = s.dgl_residual().copy()
    for _ in range(10):
        s.step()
    drift = np.abs(s.dgl_residual() - r0).max()
    assert drift <= 1e-12 * max(np.abs(r0).max(), abs(s.q_src))


def test_walk_reaches_the_straight_line_endpoint(cavity):
    """Force-free particles: whatever cells the walk crosses, the final position equals
    (z + v_z dt, sqrt((rho + v_rho dt)^2 + (v_phi dt)^2))."""
    s = _fresh(cavity)
    s.create(0.5 * s.dt_max)
    dt = s.dt = 12 * s.dt_max          # several cells per step; the fields stay zero
    m = s.mesh
    z, r, ur, up, uz = W.uniform_in_mesh(m.nodes, m.tris, 2000, 5, sigma_u=2.0)
    s.inject(z, r, ur, up, uz, -1.0, 1.0, 1e-3)
    gam = np.sqrt(1.0 + (ur ** 2 + up ** 2 + uz ** 2))
    ze = z + uz / gam * dt
    re = np.hypot(r + ur / gam * dt, up / gam * dt)
    s.push_particles(s.field_b_half())
    live = s.tri >= 0
    zn, rn = s.positions()
    assert np.allclose(zn, ze[live], atol=1e-12) and np.allclose(rn, re[live], atol=1e-12)
    # absorbed particles are exactly those whose endpoint left the cavity (0<z<1, rho<0.5)
    out = (ze <= 0) | (ze >= 1) | (re >= 0.5)
    assert np.array_equal(~live, out)
    assert s.counters[2] > 4000


def test_rotate_back_reflects_at_axis(cavity):
    """A particle crossing rho = 0 in Cartesian space reappears at |rho + v_rho dt| with
    u_rho reversed: the perfectly reflecting axis of Sec. 5.1."""
    s = _fresh(cavity)
    dt = 0.5 * s.dt_max
    s.create(dt)
    v = -0.5
    gam = 1.0 / math.sqrt(1 - v * v)
    rho0 = 0.3 * abs(v) * dt
    s.inject([0.5], [rho0], [gam * v], [0.0], [0.0], -1.0, 1.0, 1e-3)
    s.step()
    zn, rn = s.positions()
    assert abs(rn[0] - abs(rho0 + v * dt)) < 1e-14 and abs(zn[0] - 0.5) < 1e-14
    assert abs(s.u[0, 0] + gam * v) < 1e-14


def test_boris_gyration_closed_form():
    """Uniform B_z, no E: Boris turns U = u_x + i u_y by exp(-2i atan(q dt B / 2 m gamma))
    per step, and X_{n+1} = X_n + dt U_{n+1/2} / gamma (Eq. DNE) in the Cartesian plane
    of the ring; the oracle's (rho, u_rho, u_phi) must follow |X_n| and the rotated U."""
    nodes, tris, be, bt = W.rect_mesh(1.0, 1.0, 400, 21)
    s = OracleSim(nodes, tris, be, bt)
    dt, B, q, mass = 0.05, 2.0, -1.0, 1.0
    s.create(0.5 * s.dt_max, bz=B)
    s.dt = dt                       # particle-only steps: the fields stay zero
    u0 = np.array([0.03, 0.1, 0.02])          # (u_rho, u_phi, u_z)
    rho0, z0 = 0.5, 0.3
    s.inject([z0], [rho0], [u0[0]], [u0[1]], [u0[2]], q, mass, 1e-6)
    gam = math.sqrt(1 + u0 @ u0)
    theta = -2.0 * math.atan(q * dt * B / (2 * mass * gam))
    U = u0[0] + 1j * u0[1]
    X = rho0 + 0j
    for n in range(40):
        s.push_particles(s.field_b_half())
        U = U * np.exp(1j * theta)
        X = X + dt * U / gam
        zn, rn = s.positions()
        assert abs(rn[0] - abs(X)) < 1e-13
        assert abs(zn[0] - (z0 + (n + 1) * dt * u0[2] / gam)) < 1e-13
        ul = U * np.exp(-1j * np.angle(X))
        assert abs(s.u[0, 0] - ul.real) < 1e-14 and abs(s.u[0, 1] - ul.imag) < 1e-14


@pytest.mark.parametrize("component", [0, 1])
def test_uniform_E_kick(cavity, component):
    """Whitney 1-forms reproduce a constant field exactly; with edge DOFs equal to the
    line integral of a uniform E (along the low -> high orientation of App. D), B = 0,
    the Boris push adds q E dt / m to u every step exactly (Eq. DLE)."""
    s = _fresh(cavity)
    m = s.mesh
    dt = 0.5 * s.dt_max
    s.create(dt)
    E0 = 0.02
    d = m.nodes[m.edge_nodes[:, 1]] - m.nodes[m.edge_nodes[:, 0]]
    s.set_fields(E0 * d[:, component], np.zeros(m.N2))
    rng = np.random.default_rng(1)
    n = 50
    z = rng.uniform(0.3, 0.7, n)
    r = rng.uniform(0.15, 0.35, n)
    s.inject(z, r, np.zeros(n), np.zeros(n), np.zeros(n), -1.0, 1.0, 1e-9)
    # one push with the prescribed field, no field update
    Bh = s.field_b_half()
    s.push_particles(Bh)
    kick = -1.0 * E0 * dt
    uz_expected = kick if component == 0 else 0.0
    ur_expected = kick if component == 1 else 0.0
    assert np.allclose(s.u[:, 2], uz_expected, atol=1e-15)
    assert np.allclose(s.u[:, 0], ur_expected, atol=1e-15)


def test_rest_particle_is_inert(cavity):
    s = _fresh(cavity)
    s.create(0.5 * s.dt_max)
    z, r, *_ = W.uniform_in_mesh(s.mesh.nodes, s.mesh.tris, 100, 9)
    z0 = np.zeros(100)
    s.inject(z, r, z0, z0, z0, -1.0, 1.0, 1e-3)
    Q0 = s.Q.copy()
    lam0 = s.lam.copy()
    s.step()
    assert np.all(s.J == 0) and np.allclose(s.Q, Q0, atol=1e-18) and np.allclose(s.lam, lam0, atol=1e-15)


def test_energy_balance_fixes_ring_normalisation():
    """The 2D equations are the 3D ones divided by 2 pi (the Hodge integrals drop the
    azimuthal integral, App. B), so a ring of charge q drives J with q/(2 pi).  Then the
    field energy gained, times 2 pi, equals the kinetic energy lost; a missing or doubled
    2 pi would put the ratio near 2 pi or 1/(2 pi)."""
    nodes, tris, be, bt = W.rect_mesh(1.0, 1.0, 3000, 7)
    s = OracleSim(nodes, tris, be, bt)
    s.create(0.5 * s.dt_max)
    rng = np.random.default_rng(1)
    n = 20000
    z = rng.uniform(0.4, 0.6, n)
    r = np.sqrt(rng.uniform(0.3 ** 2, 0.5 ** 2, n))
    ur, up, uz = W.maxwellian(n, 0.05, rng, drift=(0.0, 0.0, 0.2))
    s.inject(z, r, ur, up, uz, -1.0, 1.0, 1e-3)
    fe0, ke0 = s.field_energy(), s.kinetic_energy()
    s.step(45)
    assert s.counters[0] == 0
    ratio = -2 * math.pi * (s.field_energy() - fe0) / (s.kinetic_energy() - ke0)
    assert abs(ratio - 1.0) < 0.02


def test_absorbed_charge_enters_dce(cavity):
    """A particle driven into the PEC wall is removed; its charge is booked at its wall
    position, and Eq. DCE holds with that sink."""
    s = _fresh(cavity)
    dt = 0.5 * s.dt_max
    s.create(dt)
    v = 0.9
    gam = 1 / math.sqrt(1 - v * v)
    s.inject([0.5], [0.5 - 0.3 * v * dt], [gam * v], [0.0], [0.0], -1.0, 1.0, 1e-3)
    s.step()
    assert s.tri[0] == -1 and s.counters[0] == 1
    assert abs(s.Qabs.sum() - s.q_src) < 1e-15
    assert np.abs(s.dce_residual()).max() * dt < 1e-15
    assert np.all(s.Q == 0)


def test_rotational_field_fixes_faraday_sign_and_time_centred_B():
    """E = (a/2)(-rho, z) in (E_z, E_rho) is a rotation field, which Whitney 1-forms
    reproduce exactly (App. A), with (curl E)_phi = dE_rho/dz - dE_z/drho = a.  Faraday's
    law then raises B_phi by -a dt per step on every face away from the walls (Eq.
    full_d_dfl; B_phi = B_f / A, Sec. 3.2).  A particle moving in the meridian plane feels
    E at its position and the time-centred B_phi = B0 - a dt / 2, and its new momentum
    must solve Boris's form of Eq. DLE: u1 - u0 = 2h (E + (u0 + u1) / (2 gamma(u0 + h E))
    x B) with h = q dt / (2 m).  This fixes the orientation of D_curl against +phi, the
    1/A of the 2-form, the averaging of B and the gathered E together."""
    nodes, tris, be, bt = W.rect_mesh(1.0, 1.0, 600, 21)
    s = OracleSim(nodes, tris, be, bt)
    m = s.mesh
    dt = 0.5 * s.dt_max
    s.create(dt)
    a, B0 = 3.0, 2.0

    def field(z, r):
        return np.stack([-0.5 * a * r, 0.5 * a * z], -1)          # (E_z, E_rho)

    pt, ph = m.nodes[m.edge_nodes[:, 0]], m.nodes[m.edge_nodes[:, 1]]
    E = np.einsum("ed,ed->e", field(*(0.5 * (pt + ph)).T), ph - pt)   # exact for linear E
    s.set_fields(E, B0 * m.area)
    Bh = s.field_b_half()
    away = ~np.any(m.edge_tag[m.tri_edges] == 1, axis=1)
    assert away.sum() > m.N2 // 2
    assert np.allclose(Bh[away] / m.area[away], B0 - a * dt, rtol=0, atol=1e-12)

    z0, r0 = 0.47, 0.53
    u0 = np.array([0.3, 0.0, 0.6])                                  # (u_rho, u_phi, u_z)
    q, mass = -1.0, 1.0
    s.inject([z0], [r0], [u0[0]], [u0[1]], [u0[2]], q, mass, 1e-9)
    assert away[s.tri[0]]
    s.push_particles(Bh)
    u1 = s.u[0]
    Ez, Er = field(z0, r0)
    Ef = np.array([Er, 0.0, Ez])
    Bf = np.array([0.0, B0 - 0.5 * a * dt, 0.0])
    h = q * dt / (2 * mass)
    gm = math.sqrt(1.0 + np.sum((u0 + h * Ef) ** 2))
    rhs = 2 * h * (Ef + np.cross(0.5 * (u0 + u1) / gm, Bf))
    assert abs(u1[1]) < 1e-15
    assert np.abs(u1 - u0 - rhs).max() < 1e-13
    # the magnetic part is not negligible: B_phi at n+1/2 alone would miss by far more
    Bn = np.array([0.0, B0 - a * dt, 0.0])
    assert np.abs(u1 - u0 - 2 * h * (Ef + np.cross(0.5 * (u0 + u1) / gm, Bn))).max() > 1e-6


def _path_current(m, r0, r1):
    """int W1_e . dr along the straight segment r0 -> r1, cell by cell: the cuts where it
    meets any mesh edge (brute force over all edges), the containing triangle of each
    piece by point location, and a 2-point Gauss rule on each piece (exact: W1 is linear
    inside a triangle), with gradients and lambda from linear solves."""
    a, b = m.nodes[m.edge_nodes[:, 0]], m.nodes[m.edge_nodes[:, 1]]
    d, e, w = r1 - r0, b - a, a - r0
    det = e[:, 0] * d[1] - d[0] * e[:, 1]            # of [d, -e] (s, t) = w
    ok = np.abs(det) > 1e-14
    sd = np.where(ok, det, 1.0)
    s = (e[:, 0] * w[:, 1] - w[:, 0] * e[:, 1]) / sd
    t = (d[0] * w[:, 1] - w[:, 0] * d[1]) / sd
    cut = ok & (s > 0) & (s < 1) & (t >= 0) & (t <= 1)
    ss = np.concatenate([[0.0], np.sort(s[cut]), [1.0]])
    x, wq = np.polynomial.legendre.leggauss(2)
    x, wq = 0.5 * (x + 1), 0.5 * wq
    J = np.zeros(m.N1)
    for s0, s1 in zip(ss[:-1], ss[1:]):
        if s1 - s0 < 1e-13:
            continue
        mid = r0 + 0.5 * (s0 + s1) * d
        tri, _ = TPart.locate(m, [mid[0]], [mid[1]])
        T = int(tri[0])
        p = m.nodes[m.tris[T]]
        G = _grad_by_solve(p)
        for xi, wi in zip(x, wq):
            r = r0 + (s0 + xi * (s1 - s0)) * d
            lam = _lam_by_solve(p, r[0], r[1])
            for k in range(3):
                ta, hb = m.edge_tail_head(T, k)
                J[m.tri_edges[T, k]] += wi * (s1 - s0) * (lam[ta] * G[hb] - lam[hb] * G[ta]) @ d
    return J


def test_multi_cell_current_is_the_line_integral_over_the_crossed_cells(cavity):
    """Eq. current summed over the pieces of a path that crosses several cells: for
    force-free particles on straight meridian paths (u_phi = 0), J must equal (q/dt) times
    the line integral of the piecewise Whitney 1-forms, computed here cell by cell from
    the path's exact cuts with the mesh edges."""
    s = _fresh(cavity)
    m = s.mesh
    s.create(0.5 * s.dt_max)
    dt = s.dt = 0.5                      # particle-only step; the fields stay zero
    rng = np.random.default_rng(21)
    n = 30
    r0 = np.stack([rng.uniform(0.1, 0.9, n), rng.uniform(0.08, 0.42, n)], 1)
    ang = rng.uniform(0, 2 * np.pi, n)
    r1 = r0 + rng.uniform(0.05, 0.15, n)[:, None] * np.stack([np.cos(ang), np.sin(ang)], 1)
    r1 = np.clip(r1, [0.02, 0.02], [0.98, 0.48])
    v = (r1 - r0) / dt                   # (v_z, v_rho), |v| < c = 1
    gam = 1.0 / np.sqrt(1.0 - np.sum(v * v, 1))
    s.inject(r0[:, 0], r0[:, 1], gam * v[:, 1], np.zeros(n), gam * v[:, 0], -1.0, 1.0, 1e-3)
    s.push_particles(s.field_b_half())
    assert np.all(s.tri >= 0) and s.counters[2] > 3 * n
    zn, rn = s.positions()
    assert np.allclose(zn, r1[:, 0], atol=1e-12) and np.allclose(rn, r1[:, 1], atol=1e-12)
    ref = sum(_path_current(m, r0[i], r1[i]) for i in range(n)) * (s.q_src / dt)
    assert np.abs(s.J - ref).max() <= 1e-12 * np.abs(ref).max()


def test_locate_by_brute_force():
    """Point location (used to place injected and emitted particles): against every
    triangle's barycentric coordinates from a linear solve, the located triangle holds
    the point (all lambda >= -1e-12, sum 1, reproducing the point) and has the largest
    smallest coordinate; points outside the mesh get -1.  On interior edge midpoints the
    answer is one of the edge's two triangles."""
    m = Mesh(*W.cavity_mesh(n_tri=300, seed=13))
    rng = np.random.default_rng(5)
    n = 1500
    z = rng.uniform(-0.1, 1.1, n)
    r = rng.uniform(0.0, 0.6, n)
    A = np.stack([np.ones((m.N2, 3)), m.nodes[m.tris][:, :, 0], m.nodes[m.tris][:, :, 1]], 1)
    Ainv = np.linalg.inv(A)                                   # lambda = Ainv @ (1, z, rho)
    lam_all = np.einsum("tij,nj->nti", Ainv, np.stack([np.ones(n), z, r], 1))
    mins = lam_all.min(2)
    inside = mins.max(1) >= -1e-12
    tri, lam = TPart.locate(m, z, r)
    assert np.array_equal(tri >= 0, inside)
    k = np.flatnonzero(inside)
    assert np.array_equal(tri[k], np.argmax(mins[k], 1))
    assert np.allclose(lam[k], lam_all[k, tri[k]], rtol=0, atol=1e-12)
    assert np.allclose(lam[k].sum(1), 1.0, atol=1e-14)
    p = m.nodes[m.tris[tri[k]]]
    assert np.allclose(np.einsum("nk,nkd->nd", lam[k], p), np.stack([z[k], r[k]], 1), atol=1e-14)
    inner = np.flatnonzero(m.edge_tag == 0)
    mid = m.nodes[m.edge_nodes[inner]].mean(1)
    tri_e, lam_e = TPart.locate(m, mid[:, 0], mid[:, 1])
    assert np.all((tri_e == m.edge_tris[inner, 0]) | (tri_e == m.edge_tris[inner, 1]))
    assert lam_e.min() >= -1e-12


def test_kinetic_energy_limits(cavity):
    """Kinetic energy of the macro-particles: zero at rest, w m u^2 / 2 for u << c and
    w m c |u| for u >> c (per macro-particle of weight w; c = 1 here)."""
    z, r, *_ = W.uniform_in_mesh(cavity.mesh.nodes, cavity.mesh.tris, 1, 2)
    w, mass = 3e-3, 2.0
    for u, expect, tol in ((0.0, 0.0, 0.0), (1e-4, w * mass * 1e-8 / 2, 1e-6),
                           (1e4, w * mass * 1e4, 1e-4)):
        s = _fresh(cavity)
        s.create(0.5 * s.dt_max)
        s.inject(z, r, [0.0], [u], [0.0], -1.0, mass, w)
        assert abs(s.kinetic_energy() - expect) <= tol * expect


def test_walk_cap_removes_the_particle_and_books_its_charge(cavity):
    """A particle whose step crosses more cells than the walk cap (16 crossings) is taken
    out where the cap is reached: it counts as a walk-cap overflow, its charge is booked
    as removed at that point, and Eq. DCE holds with that sink.  A slower particle on the
    same line, crossing fewer cells, arrives."""
    out = {}
    for frac in (0.9, 0.05):
        s = _fresh(cavity)
        s.create(0.5 * s.dt_max)
        dt = s.dt = 1.0                       # particle-only step; the fields stay zero
        v = frac * 0.8 / dt                   # along z across most of the cavity
        gam = 1.0 / math.sqrt(1.0 - v * v)
        s.inject([0.1], [0.23], [0.0], [0.0], [gam * v], -1.0, 1.0, 1e-3)
        Qn = s.push_particles(s.field_b_half())
        s.Q_prev, s.Q = s.Q, Qn
        out[frac] = (s.tri[0], s.counters.copy())
        assert np.abs(s.dce_residual()).max() * dt < 1e-15
        if frac == 0.9:
            assert abs(s.Qabs.sum() - s.q_src) < 1e-15 and np.all(Qn == 0)
    assert out[0.9][0] == -1 and out[0.9][1][0] == 1 and out[0.9][1][1] == 1
    assert out[0.9][1][2] == TPart.WALK_CAP
    assert out[0.05][0] >= 0 and out[0.05][1][1] == 0 and 0 < out[0.05][1][2] < TPart.WALK_CAP


def test_openmp_build_matches_the_plain_build(cavity):
    """The timed CPU baseline runs particles.c built with -fopenmp (all host cores, atomic
    sums).  Each particle's arithmetic is the same code, so positions, momenta, triangles
    and counters agree exactly with the plain build; J, Q and Q_abs agree up to the order
    of their sums."""
    if TPart.build_oracle_omp_lib() is None:
        pytest.skip("gcc without OpenMP")
    m = cavity.mesh
    pm = TPart.PushMesh(m)
    rng = np.random.default_rng(5)
    E = rng.uniform(-0.05, 0.05, m.N1)
    Bavg = rng.uniform(-1e-3, 1e-3, m.N2)
    z, r, ur, up, uz = W.uniform_in_mesh(m.nodes, m.tris, 20_000, 6, sigma_u=0.8)
    tri0, lam0 = TPart.locate(m, z, r)
    u0 = np.stack([ur, up, uz], 1)
    out = []
    for threads in (False, True):
        tri, lam, u = tri0.astype(np.int32).copy(), lam0.copy(), u0.copy()
        J, Q, Qa = np.zeros(m.N1), np.zeros(m.N0), np.zeros(m.N0)
        cnt = TPart.push(pm, E, Bavg, 0.3, 0.5 * cavity.dt_max, -1.0, 1.0, 1e-3, tri, lam, u,
                         J, Q, Qa, threads=threads)
        out.append((tri, lam, u, J, Q, Qa, cnt))
    a, b = out
    for x, y in zip(a[:3] + a[6:], b[:3] + b[6:]):
        assert np.array_equal(x, y)
    assert a[6][2] > 0 and a[6][0] > 0
    for x, y in zip(a[3:6], b[3:6]):
        assert np.abs(x - y).max() <= 1e-12 * np.abs(x).max()
    assert TPart.host_threads(True) >= 1 and TPart.host_threads(False) == 1
