"""Output-port power recorded on the device (pic_sim_set_ports) against the oracle's
Poynting flux of its own fields (oracle/port.py), step by step, both builds, with the
steps replayed as CUDA graphs: two planes across a guide, E^n and the time-centred
B_phi of each step."""
import numpy as np
import pytest

import workloads as W
from oracle import OracleSim
from oracle import port as OPort

pytestmark = pytest.mark.gpu

PORTS = [(0.4321, 0.0, 0.5), (0.6113, 0.1, 0.37)]


@pytest.fixture(scope="module")
def pic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import pic as p
    return p


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_port_power_matches_the_oracle(pic, precision, tol):
    arrays = W.rect_mesh(1.0, 0.5, 1200, 17)
    o = OracleSim(*arrays)
    m = o.mesh
    dt = 0.5 * o.dt_max
    o.create(dt)
    E0 = W.random_edge_values(m.N1, 0.05, 41)
    B0 = W.random_edge_values(m.N2, 1e-3, 42)
    o.set_fields(E0, B0)
    prec = pic.PIC_FP64 if precision == "fp64" else pic.PIC_FP32
    mesh = pic.pic_mesh_create(*arrays, precision=prec)
    pic.pic_spai_build(mesh)
    sim = pic.pic_sim_create(mesh, dt, 0.0, 16)
    pic.pic_sim_set_sort_interval(sim, 2)
    pic.pic_sim_set_graph(sim, True)
    pic.pic_fields_set(sim, E0, B0)
    z, r0, r1 = (np.array(v) for v in zip(*PORTS))
    steps = 12
    pic.pic_sim_set_ports(sim, z, r0, r1, capacity=steps + 4, every=1)
    pic.pic_step(sim, steps)
    rec, dropped = pic.pic_ports_read(sim)
    assert rec.shape == (steps, len(PORTS)) and dropped == 0
    ref = np.zeros((steps, len(PORTS)))
    for k in range(steps):
        Bavg = 0.5 * (o.field_b_half() + o.B)
        for j, (zz, a, b) in enumerate(PORTS):
            ref[k, j] = OPort.port_power(m, o.E, Bavg, zz, a, b)
        o.step()
    for j in range(len(PORTS)):
        scale = np.abs(ref[:, j]).max()
        assert scale > 0
        assert np.abs(rec[:, j] - ref[:, j]).max() <= tol * scale, (j, rec[:, j], ref[:, j])
    # records are consumed by a read; the step phase carries on
    pic.pic_step(sim, 3)
    rec2, _ = pic.pic_ports_read(sim)
    assert rec2.shape == (3, len(PORTS))
    with pytest.raises(pic.PicError) as e:
        pic.pic_sim_set_ports(sim, [1.5], [0.0], [0.5], capacity=4)   # outside the mesh
    assert e.value.status == pic.PIC_ERR_ARG
    pic.pic_sim_set_ports(sim, None, None, None, capacity=1)
