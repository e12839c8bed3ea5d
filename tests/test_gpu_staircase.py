"""Staircasing (Sec. 5.3): the pi-point frequency of one slow-wave-structure period from
the GPU field solver converges on conformal meshes, and staircased meshes of the same
spacing underestimate it by more than the conformal meshes miss it; the field update on a
staircased mesh matches the oracle."""
import numpy as np
import pytest

import workloads as W
from workloads.bwo import EPS0, MU0, C0
from workloads.meshes import sws_cell_mesh
from oracle import OracleSim

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import pic as p
    return p


def test_staircased_field_update_matches_oracle(pic):
    nodes, tris, be, bt = sws_cell_mesh(1000, staircase=True)
    o = OracleSim(nodes, tris, be, bt, eps0=EPS0, mu0=MU0, c=C0)
    m = o.mesh
    dt = 0.5 * o.dt_max
    o.create(dt)
    E0 = W.tm0np_edge_dofs(m.nodes, m.edge_nodes, 15e-3, 7.5e-3, 1, 1)
    o.set_fields(E0, np.zeros(m.N2))
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, eps0=EPS0, mu0=MU0, c=C0,
                               precision=pic.PIC_FP64)
    pic.pic_spai_build(mesh)
    sim = pic.pic_sim_create(mesh, dt, 0.0, 16)
    pic.pic_fields_set(sim, E0, np.zeros(m.N2))
    pic.pic_step(sim, 200)
    o.step(200)
    E, B = pic.pic_fields_get(sim)
    assert np.abs(E - o.E).max() <= 1e-11 * np.abs(o.E).max()
    assert np.abs(B - o.B).max() <= 1e-11 * np.abs(o.B).max()


def test_staircasing_underestimates_the_pi_point(pic):
    from paper_1701_03784_gb300 import coldtest
    conf = {n: coldtest.ring_down(n, False)[1] for n in (1000, 2000, 4000, 8000)}
    stair = {n: coldtest.ring_down(n, True)[1] for n in (1000, 2000, 4000)}
    ref = conf[8000]
    for n in (1000, 2000, 4000):
        assert abs(conf[n] / ref - 1.0) < 1e-3, (n, conf[n], ref)
        assert stair[n] < ref * (1.0 - 5e-4), (n, stair[n], ref)
        assert abs(stair[n] / ref - 1.0) > abs(conf[n] / ref - 1.0)
