"""The field update with the SPAI patterns and drop tolerances of the sweep (Sec. 3.1
leaves both open): 200 leapfrog steps of the cavity modes on the GPU (FP64 build) against
the oracle run with its own M of the same pattern and tolerance."""
import numpy as np
import pytest

import workloads as W
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


@pytest.mark.parametrize("level,tau", [(1, 1e-4), (2, 1e-2), (3, 1e-4)])
def test_field_update_matches_oracle_across_the_sweep(pic, level, tau):
    nodes, tris, be, bt = W.cavity_mesh()
    o = OracleSim(nodes, tris, be, bt, level=level, drop_tol=tau)
    m = o.mesh
    dt = 0.5 * o.dt_max
    o.create(dt)
    E0 = (W.tm0np_edge_dofs(m.nodes, m.edge_nodes, 0.5, 1.0, 1, 0)
          + W.tm0np_edge_dofs(m.nodes, m.edge_nodes, 0.5, 1.0, 1, 1))
    o.set_fields(E0, np.zeros(m.N2))
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, precision=pic.PIC_FP64)
    dt_max = pic.pic_spai_build(mesh, level, tau)
    assert abs(dt_max - o.dt_max) <= 1e-9 * o.dt_max
    sim = pic.pic_sim_create(mesh, dt, 0.0, 16)
    pic.pic_fields_set(sim, E0, np.zeros(m.N2))
    for _ in range(4):
        pic.pic_step(sim, 50)
        o.step(50)
        E, B = pic.pic_fields_get(sim)
        assert np.abs(E - o.E).max() <= 1e-11 * np.abs(o.E).max()
        assert np.abs(B - o.B).max() <= 1e-11 * np.abs(o.B).max()
    pic.pic_sim_destroy(sim)
    pic.pic_mesh_destroy(mesh)
