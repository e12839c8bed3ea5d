"""The absorbing layer on the GPU (pic_sim_set_loss, the stand-in for the paper's PML,
Sec. 5.3): fields against the oracle's lossy update step by step, and the guided pulse
taken up by a graded layer."""
import numpy as np
import pytest

import workloads as W
from oracle import OracleSim
from paper_1701_03784_gb300 import ports

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


@pytest.fixture(scope="module")
def guide():
    arrays = W.meshes.rect_mesh(16.0, 1.0, 6000, 21)
    return arrays, OracleSim(*arrays)


def _pulse(m):
    zc = 0.5 * (m.nodes[m.edge_nodes[:, 0], 0] + m.nodes[m.edge_nodes[:, 1], 0])
    return (W.tm0np_edge_dofs(m.nodes, m.edge_nodes, 1.0, 16.0, 1, 30)
            * np.exp(-((zc - 5.0) / 1.5) ** 2))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_lossy_fields_match_oracle(pic, guide, prec):
    """A pulse already inside a graded layer (strong conductivities) for 40 steps, with
    charged particles in the guide: E and B against the oracle (FP64 1e-12 per step,
    FP32 1e-4), and the Gauss-law drift outside the layer at round-off."""
    arrays, oracle = guide
    o = OracleSim.__new__(OracleSim)
    o.__dict__.update({k: (v.copy() if isinstance(v, np.ndarray) else v)
                       for k, v in oracle.__dict__.items()})
    m = o.mesh
    dt = 0.5 * o.dt_max
    o.create(dt, bz=0.5)
    E0 = _pulse(m)
    o.set_fields(E0, np.zeros(m.N2))
    se, sm = ports.graded_layer(m.nodes, m.edge_nodes, m.tris, 3.0, 8.0,
                                ports.sigma_max_for(1e-6, 5.0, 3))
    o.set_loss(se, sm)
    z, r, ur, up, uz = W.uniform_in_mesh(arrays[0], m.tris, 4000, 5, sigma_u=0.3)
    keep = z > 9.0
    o.inject(z[keep], r[keep], ur[keep], up[keep], uz[keep], -1.0, 1.0, 1e-3)
    P = pic.PIC_FP64 if prec == "fp64" else pic.PIC_FP32
    mesh = pic.pic_mesh_create(*arrays, precision=P)
    pic.pic_spai_build(mesh)
    sim = pic.pic_sim_create(mesh, dt, 0.5, 10_000)
    pic.pic_fields_set(sim, E0, np.zeros(m.N2))
    pic.pic_sim_set_loss(sim, se, sm)
    pic.pic_particles_inject(sim, z[keep], r[keep], ur[keep], up[keep], uz[keep], -1.0, 1.0, 1e-3)
    steps = 40
    pic.pic_step(sim, steps)
    o.step(steps)
    d = pic.pic_diagnostics(sim, fields=True)
    tol = 1e-12 * steps if prec == "fp64" else 1e-4
    assert np.abs(d["E"] - o.E).max() <= tol * np.abs(E0).max()
    assert np.abs(d["B"] - o.B).max() <= tol * np.abs(o.B).max()
    assert d["dgl_drift"] < (1e-10 if prec == "fp64" else 1e-5)
    pic.pic_sim_destroy(sim)
    pic.pic_mesh_destroy(mesh)


def test_graded_layer_absorbs_a_guided_pulse_on_the_gpu(pic, guide):
    arrays, oracle = guide
    m = oracle.mesh
    mesh = pic.pic_mesh_create(*arrays, precision=pic.PIC_FP32)
    dt = 0.5 * pic.pic_spai_build(mesh)
    E0 = _pulse(m)
    left = {}
    for layer in (False, True):
        sim = pic.pic_sim_create(mesh, dt, 0.0, 16)
        pic.pic_fields_set(sim, E0, np.zeros(m.N2))
        if layer:
            pic.pic_sim_set_loss(sim, *ports.graded_layer(
                m.nodes, m.edge_nodes, m.tris, 12.0, 16.0, ports.sigma_max_for(1e-4, 4.0, 3)))
        e0 = pic.pic_diagnostics(sim)["field_energy"]
        pic.pic_step(sim, int(30.0 / dt))
        left[layer] = pic.pic_diagnostics(sim)["field_energy"] / e0
        pic.pic_sim_destroy(sim)
    assert left[False] > 0.95 and left[True] < 0.01
    pic.pic_mesh_destroy(mesh)


def test_removing_the_layer_restores_the_lossless_update(pic, guide):
    """A layer set and then removed before any step leaves the fields bit-identical to a
    simulation that never had one (FP32), and the probes of a simulation can be removed."""
    arrays, oracle = guide
    m = oracle.mesh
    mesh = pic.pic_mesh_create(*arrays, precision=pic.PIC_FP32)
    dt = 0.5 * pic.pic_spai_build(mesh)
    E0 = _pulse(m)
    out = []
    for layer in (False, True):
        sim = pic.pic_sim_create(mesh, dt, 0.0, 16)
        pic.pic_fields_set(sim, E0, np.zeros(m.N2))
        if layer:
            pic.pic_sim_set_loss(sim, *ports.graded_layer(
                m.nodes, m.edge_nodes, m.tris, 12.0, 16.0, ports.sigma_max_for(1e-4, 4.0, 3)))
            pic.pic_sim_set_loss(sim, None, None)
            pic.pic_sim_set_probes(sim, [0, 1], [0, 0], [1.0, 1.0], [2], capacity=8, every=1)
            pic.pic_sim_set_probes(sim, [], [], [], [], capacity=8, every=1)
        pic.pic_step(sim, 50)
        out.append(pic.pic_fields_get(sim))
        if layer:
            with pytest.raises(pic.PicError) as e:
                pic.pic_probes_read(sim)
            assert e.value.status == pic.PIC_ERR_STATE
        pic.pic_sim_destroy(sim)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    pic.pic_mesh_destroy(mesh)
