"""Device-recorded field probes (pic_sim_set_probes): the recorded sums equal the same
sums taken on the host from the fields read back after each step, with and without CUDA
graph replay, and the buffer's capacity rule."""
import numpy as np
import pytest

import workloads as W

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


def _sim(pic, prec, graph):
    nodes, tris, be, bt = W.cavity_mesh()
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, precision=prec)
    dt = 0.5 * pic.pic_spai_build(mesh)
    info = pic.pic_mesh_info(mesh)
    sim = pic.pic_sim_create(mesh, dt, 0.3, 40_000)
    pic.pic_sim_set_sort_interval(sim, 3)
    pic.pic_sim_set_graph(sim, graph)
    pic.pic_fields_set(sim, W.random_edge_values(info["n_edges"], 0.05, 1), np.zeros(info["n_tris"]))
    z, r, ur, up, uz = W.uniform_in_mesh(nodes, tris, 20_000, 2, sigma_u=0.5)
    pic.pic_particles_inject(sim, z, r, ur, up, uz, -1.0, 1.0, 1e-3)
    return mesh, sim, info["n_tris"]


@pytest.mark.parametrize("prec,graph", [("fp64", False), ("fp32", False), ("fp32", True)])
def test_probes_match_host_sums(pic, prec, graph):
    P = pic.PIC_FP64 if prec == "fp64" else pic.PIC_FP32
    rng = np.random.default_rng(5)
    mesh, sim, n2 = _sim(pic, P, graph)
    groups = [rng.choice(n2, 300, replace=False), rng.choice(n2, 1, replace=False),
              np.arange(n2)]
    weights = [rng.uniform(0.5, 2.0, len(g)) for g in groups]
    power = [2, 1, 2]
    face = np.concatenate(groups)
    group = np.concatenate([np.full(len(g), k) for k, g in enumerate(groups)])
    pic.pic_sim_set_probes(sim, face, group, np.concatenate(weights), power, capacity=64,
                           every=3)
    pic.pic_step(sim, 30)
    rec, dropped = pic.pic_probes_read(sim)
    assert rec.shape == (10, 3) and dropped == 0
    # the same 30 steps, one at a time, on a fresh simulation: B after step s (0-based)
    mesh2, sim2, _ = _sim(pic, P, False)
    host = []
    for s in range(30):
        pic.pic_step(sim2, 1)
        if s % 3 == 0:
            B = pic.pic_fields_get(sim2)[1]
            host.append([np.sum(w * (B[g] ** p)) for g, w, p in zip(groups, weights, power)])
    host = np.array(host)
    assert np.allclose(rec, host, rtol=1e-12, atol=0)
    # records are consumed by a read; the phase carries on
    pic.pic_step(sim, 6)
    rec2, _ = pic.pic_probes_read(sim)
    assert len(rec2) == 2


def test_probe_capacity(pic):
    mesh, sim, n2 = _sim(pic, pic.PIC_FP32, False)
    pic.pic_sim_set_probes(sim, np.arange(10), np.zeros(10), np.ones(10), [1], capacity=4,
                           every=1)
    pic.pic_step(sim, 7)
    rec, dropped = pic.pic_probes_read(sim)
    assert len(rec) == 4 and dropped == 3
    with pytest.raises(pic.PicError) as e:
        pic.pic_sim_set_probes(sim, [n2], [0], [1.0], [1], capacity=4, every=1)
    assert e.value.status == pic.PIC_ERR_ARG
