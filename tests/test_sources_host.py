"""The library's static-field solve (pic_static_potential, host code) against the oracle's
Laplace problem on the same mesh and held potentials.  CPU only."""
import numpy as np
import pytest

import workloads as W
from oracle import sources as S
from oracle.operators import Mesh, hodge_eps


@pytest.fixture(scope="module")
def pic():
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import pic as p
    return p


@pytest.mark.parametrize("case", ["planar", "quadrupole", "diode_si", "charged"])
def test_static_potential_matches_oracle(pic, case):
    if case == "diode_si":
        nodes, tris, be, bt = W.diode_mesh(n_tri=3000, seed=8)
        eps0 = 8.8541878128e-12
    else:
        nodes, tris, be, bt = W.cavity_mesh(a=0.5, L=1.0, n_tri=1200, seed=9)
        eps0 = 1.0
    om = Mesh(nodes, tris, be, bt)
    if case == "quadrupole":
        held = np.flatnonzero(om.node_on_pec)
        vals = om.nodes[held, 1] ** 2 - 2.0 * (om.nodes[held, 0] - 0.5) ** 2
    else:
        z = om.nodes[:, 0]
        held = np.flatnonzero((z == z.min()) | (z == z.max()))
        vals = np.where(om.nodes[held, 0] == z.min(), 0.0, 1e5)
    Q = None
    if case == "charged":
        Q = np.random.default_rng(4).normal(size=om.N0) * 0.1
    phi_o, E_o = S.static_potential(om, hodge_eps(om, eps0), held, vals, charge=Q)
    m = pic.pic_mesh_create(nodes, tris, be, bt, eps0=eps0, mu0=1.0 if eps0 == 1.0 else 1.25663706212e-6)
    phi, E = pic.pic_static_potential(m, held, vals, charge=Q)
    scale = np.abs(phi_o).max()
    assert np.abs(phi - phi_o).max() <= 1e-9 * scale
    assert np.abs(E - E_o).max() <= 1e-9 * scale
    pic.pic_mesh_destroy(m)


def test_static_potential_errors(pic):
    nodes, tris, be, bt = W.cavity_mesh(a=0.5, L=1.0, n_tri=300, seed=9)
    m = pic.pic_mesh_create(nodes, tris, be, bt)
    with pytest.raises(pic.PicError) as e:
        pic.pic_static_potential(m, np.array([10 ** 6]), np.array([1.0]))
    assert e.value.status == pic.PIC_ERR_ARG
    with pytest.raises(pic.PicError) as e:
        pic.pic_static_potential(m, np.array([], np.int32), np.array([]))
    assert e.value.status == pic.PIC_ERR_ARG
    pic.pic_mesh_destroy(m)
