"""Bounded device waits that run out.  The particle kernel's tile pipeline (FP32 build)
waits on mbarriers with a poll limit; a test sets the limit to 0 polls so that every
such wait gives up at once.  The step must then end (no hang), the next diagnostics and
charge read-backs must report PIC_ERR_TIMEOUT, and the context must stay usable: a new
simulation afterwards steps exactly like one run before the timeout.  The surrogate
network's tensor-core inference kernel waits the same way, under its own limit."""
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


def _sim(pic, n=20_000):
    nodes, tris, be, bt = W.cavity_mesh()
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, precision=pic.PIC_FP32)
    dt = 0.5 * pic.pic_spai_build(mesh)
    sim = pic.pic_sim_create(mesh, dt, 0.3, 2 * n)
    info = pic.pic_mesh_info(mesh)
    pic.pic_fields_set(sim, W.random_edge_values(info["n_edges"], 0.05, 1),
                       W.random_edge_values(info["n_tris"], 1e-3, 2))
    z, r, ur, up, uz = W.uniform_in_mesh(nodes, tris, n, 3, sigma_u=0.3)
    pic.pic_particles_inject(sim, z, r, ur, up, uz, -1.0, 1.0, 1e-3)
    return sim


def _state(pic, sim):
    d = pic.pic_diagnostics(sim, fields=True)
    p = pic.pic_particles_get(sim)
    o = np.argsort(p["pid"])
    return d, {k: p[k][o] for k in ("tri", "lam", "u")}


def test_waits_that_run_out_are_reported_and_leave_the_context_usable(pic):
    import torch
    ref = _sim(pic)
    pic.pic_step(ref, 3)
    d_ref, p_ref = _state(pic, ref)
    assert d_ref["n_crossings"] > 0

    bad = _sim(pic)
    pic.pic_sim_set_wait_limit(bad, 0)
    pic.pic_step(bad, 2)                  # enqueued; the kernels give up and return
    torch.cuda.synchronize()
    for call in (lambda: pic.pic_diagnostics(bad),
                 lambda: pic.pic_charges_get(bad),
                 lambda: pic.pic_charges_get_static(bad, np.zeros(pic.pic_mesh_info(bad.mesh)["n_nodes"]))):
        with pytest.raises(pic.PicError) as e:
            call()
        assert e.value.status == pic.PIC_ERR_TIMEOUT
        assert "timed out" in pic.pic_last_error()
    with pytest.raises(pic.PicError):
        pic.pic_sim_set_wait_limit(bad, -1)
    del bad

    # the device and the library are fine: the same run again matches bit for bit, and
    # restoring the default bound on a new simulation changes nothing
    again = _sim(pic)
    pic.pic_sim_set_wait_limit(again, 1 << 14)
    pic.pic_step(again, 3)
    d, p = _state(pic, again)
    for k in ("tri", "lam", "u"):
        assert np.array_equal(p[k], p_ref[k]), k
    for k in ("E", "B", "J"):
        assert np.array_equal(d[k], d_ref[k]), k
    assert d["dce_nonzero"] == 0


def test_inference_waits_that_run_out_are_reported(pic):
    """The tensor-core inference kernel's waits (weight chunks, products, operands) with a
    limit of 0 polls: the forward call returns PIC_ERR_TIMEOUT instead of hanging, and with
    the default bound restored the same network gives the same outputs bit for bit."""
    import torch
    from tests.mlp_util import flat, members
    sizes, E = (6, 256, 256, 33), 3
    m = pic.pic_mlp_create(E, sizes, 256)
    pic.pic_mlp_params_set(m, np.stack([flat(W, b) for W, b in members(E, sizes, seed=41)]))
    X = torch.tensor(np.random.default_rng(42).uniform(-1, 1, (1000, 6)), dtype=torch.float32,
                     device="cuda")
    Y0 = pic.pic_mlp_forward(m, X, tensor_cores=True).cpu().numpy()
    pic.pic_mlp_set_wait_limit(m, 0)
    with pytest.raises(pic.PicError) as e:
        pic.pic_mlp_forward(m, X, tensor_cores=True)
    assert e.value.status == pic.PIC_ERR_TIMEOUT
    assert "timed out" in pic.pic_last_error()
    with pytest.raises(pic.PicError):
        pic.pic_mlp_set_wait_limit(m, -1)
    pic.pic_mlp_set_wait_limit(m, 1 << 22)
    Y1 = pic.pic_mlp_forward(m, X, tensor_cores=True).cpu().numpy()
    assert np.array_equal(Y0, Y1)
    assert np.all(np.isfinite(pic.pic_mlp_forward(m, X, tensor_cores=False).cpu().numpy()))
