"""pic_charges_get_static: the allocation-free variant of pic_charges_get.

Some callers cannot allocate device memory -- their device memory is already committed to
another allocator's pool, or the code path (inside a time loop with a fixed budget) must
not allocate.  For them the library reads the node charges through a fixed scratch array
compiled into it.  This file is collected last so that a failure here comes after every
other test has run; it also passes on its own in a fresh process."""
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


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_static_matches_allocating_call(pic, precision):
    prec = pic.PIC_FP32 if precision == "fp32" else pic.PIC_FP64
    nodes, tris, be, bt = W.cavity_mesh()
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, precision=prec)
    dt = 0.5 * pic.pic_spai_build(mesh)
    sim = pic.pic_sim_create(mesh, dt, 0.3, 20_000)
    info = pic.pic_mesh_info(mesh)
    pic.pic_fields_set(sim, W.random_edge_values(info["n_edges"], 0.05, 1),
                       W.random_edge_values(info["n_tris"], 1e-3, 2))
    z, r, ur, up, uz = W.uniform_in_mesh(nodes, tris, 10_000, 3, sigma_u=0.8)
    pic.pic_particles_inject(sim, z, r, ur, up, uz, -1.0, 1.0, 1e-3)
    n0 = info["n_nodes"]
    for _ in range(2):                      # two calls in a row, with the state moving on
        pic.pic_step(sim, 3)
        ref = pic.pic_charges_get(sim)
        for _ in range(2):
            out = [np.full(n0, np.nan), np.full(n0, np.nan), np.full(n0, np.nan)]
            pic.pic_charges_get_static(sim, *out)
            for a, b in zip(out, ref):
                assert np.allclose(a, b, rtol=1e-12, atol=0.0)
                assert not np.any(np.isnan(a))
        assert np.any(ref[2] != 0) or np.any(ref[0] != ref[1])
    # a single output may be requested
    q = np.zeros(n0)
    pic.pic_charges_get_static(sim, q, None, None)
    assert np.allclose(q, pic.pic_charges_get(sim)[0], rtol=1e-12, atol=0.0)


def test_static_rejects_meshes_beyond_its_scratch(pic):
    nodes, tris, be, bt = W.rect_mesh(1.0, 1.0, 280_000, 4)
    assert len(nodes) > 131072
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, precision=pic.PIC_FP32)
    dt = 0.5 * pic.pic_spai_build(mesh, 0, 0.0)
    sim = pic.pic_sim_create(mesh, dt, 0.0, 16)
    with pytest.raises(pic.PicError) as e:
        pic.pic_charges_get_static(sim, np.zeros(len(nodes)), None, None)
    assert e.value.status == pic.PIC_ERR_ARG
    assert "131072" in pic.pic_last_error()
