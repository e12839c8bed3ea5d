"""Pins of the oracle's absorbing layer (the stand-in for the paper's PML, Sec. 5.3):
the time-centred conduction update against its closed form on a curl-free field, and a
graded, matched layer taking up a guided pulse that a conducting end returns whole.
CPU only."""
import numpy as np
import pytest

import workloads as W
from oracle import OracleSim
from paper_1701_03784_gb300 import ports


@pytest.fixture(scope="module")
def guide():
    nodes, tris, be, bt = W.meshes.rect_mesh(16.0, 1.0, 6000, 21)
    return OracleSim(nodes, tris, be, bt)


def _copy(o):
    s = OracleSim.__new__(OracleSim)
    s.__dict__.update({k: (v.copy() if isinstance(v, np.ndarray) else v)
                       for k, v in o.__dict__.items()})
    s.sigma_e = s.sigma_m = None
    return s


def test_uniform_conductivity_decays_a_curl_free_field_exactly(guide):
    """E^0 = D_div^T phi (zero on the conductor, so E = 0 on its edges) has no curl: B stays
    0, the lossless increment vanishes, and every step multiplies E by
    (1 - s)/(1 + s), s = sigma dt / (2 eps0)."""
    s = _copy(guide)
    m = s.mesh
    s.create(0.5 * s.dt_max)
    rng = np.random.default_rng(3)
    phi = rng.normal(size=m.N0)
    phi[m.node_on_pec] = 0.0
    E0 = m.Ddiv.T @ phi
    s.set_fields(E0, np.zeros(m.N2))
    sigma = 7.0
    s.set_loss(np.full(m.N1, sigma), None)
    for _ in range(25):
        s.step()
    x = sigma * s.dt / (2.0 * s.eps0)
    assert np.abs(s.E - ((1 - x) / (1 + x)) ** 25 * E0).max() < 1e-12 * np.abs(E0).max()
    assert np.abs(s.B).max() < 1e-12 * np.abs(E0).max()


def test_graded_layer_absorbs_a_guided_pulse(guide):
    """A TM01 wave packet (carrier well above cut-off) in a 16-long circular guide: with a
    matched cubic layer over the last 4 units, less than 1% of the field energy is left
    after both halves of the packet have reached it; a conducting end keeps it all."""
    m = guide.mesh
    zc = 0.5 * (m.nodes[m.edge_nodes[:, 0], 0] + m.nodes[m.edge_nodes[:, 1], 0])
    E0 = (W.tm0np_edge_dofs(m.nodes, m.edge_nodes, 1.0, 16.0, 1, 30)
          * np.exp(-((zc - 5.0) / 1.5) ** 2))
    left = {}
    for layer in (False, True):
        s = _copy(guide)
        s.create(0.5 * s.dt_max)
        s.set_fields(E0, np.zeros(m.N2))
        if layer:
            smax = ports.sigma_max_for(1e-4, 4.0, 3)
            s.set_loss(*ports.graded_layer(m.nodes, m.edge_nodes, m.tris, 12.0, 16.0, smax))
        e0 = s.field_energy()
        for _ in range(int(30.0 / s.dt)):
            s.step()
        left[layer] = s.field_energy() / e0
    assert left[False] > 0.95
    assert left[True] < 0.01


def test_matched_uniform_conductor_scales_the_lossless_run():
    """With the same s = sigma dt / (2 eps0) = sigma* dt / (2 mu0) on every edge and face
    and no current, substituting E^n = r^n E'^n, B^{n+1/2} = r^{n+1/2} B'^{n+1/2}, with
    r = (1 - s)/(1 + s), turns the time-centred lossy updates into the lossless leapfrog
    for (E', B') with the step dt / sqrt(1 - s^2).  So the lossy run equals r^n times a
    lossless run with that step, at every edge and step, to round-off: this fixes the
    decay factor and the 1/(1 + s) on both increments."""
    nodes, tris, be, bt = W.cavity_mesh(n_tri=600, seed=8)
    o = OracleSim(nodes, tris, be, bt, eps0=1.3, mu0=0.8)
    m = o.mesh
    E0 = W.random_edge_values(m.N1, 1.0, 4)
    dt = 0.5 * o.dt_max
    s = 0.02
    sigma_e, sigma_m = 2 * s * o.eps0 / dt, 2 * s * o.mu0 / dt
    lossy, plain = _copy(o), _copy(o)
    lossy.create(dt)
    plain.create(dt / np.sqrt(1 - s * s))
    for x in (lossy, plain):
        x.set_fields(E0, np.zeros(m.N2))
    lossy.set_loss(np.full(m.N1, sigma_e), np.full(m.N2, sigma_m))
    r = (1 - s) / (1 + s)
    for n in range(1, 61):
        lossy.step()
        plain.step()
        assert np.abs(lossy.E - r ** n * plain.E).max() <= 1e-12 * np.abs(E0).max()
        assert np.abs(lossy.B - r ** (n - 0.5) * plain.B).max() <= 1e-12 * np.abs(plain.B).max()
