"""Batched ripple sweep: one simulation of the union of several BWO instances (shifted
apart along z) advances each instance as its own simulation does.  The operators of the
method are local to a mesh, so the union's are block-diagonal; the only differences are
round-off of the shifted node coordinates, hence the FP32 parity tolerance."""
import numpy as np
import pytest

from workloads.sweep import sweep_instance, union, WEIGHT
from workloads.bwo import EPS0, MU0, C0, QE, ME, BZ_BWO

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


def _mesh(pic, nodes, tris, be, bt):
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, eps0=EPS0, mu0=MU0, c=C0,
                               precision=pic.PIC_FP32)
    return mesh, pic.pic_spai_build(mesh, 2, 1e-4)


def _sim(pic, nodes, tris, be, bt, dt, z, r, ur, up, uz, steps):
    mesh, _ = _mesh(pic, nodes, tris, be, bt)
    info = pic.pic_mesh_info(mesh)
    sim = pic.pic_sim_create(mesh, dt, BZ_BWO, len(z) + 1024)
    pic.pic_sim_set_sort_interval(sim, 4)
    pic.pic_fields_set(sim, np.zeros(info["n_edges"]), np.zeros(info["n_tris"]))
    pic.pic_particles_inject(sim, z, r, ur, up, uz, QE, ME, WEIGHT)
    pic.pic_step(sim, steps)
    d = pic.pic_diagnostics(sim, fields=True)
    p = pic.pic_particles_get(sim)
    order = np.argsort(p["pid"])
    return info, d, {k: p[k][order] for k in ("pid", "tri", "lam", "u")}


def test_union_advances_each_instance_like_its_own_simulation(pic):
    ins = [sweep_instance(i, scale=0.01) for i in range(3)]
    u = union(ins)
    dt = 0.5 * _mesh(pic, u["nodes"], u["tris"], u["be"], u["bt"])[1]
    steps = 20
    info_u, du, pu = _sim(pic, u["nodes"], u["tris"], u["be"], u["bt"], dt, u["z"], u["r"],
                          u["ur"], u["up"], u["uz"], steps)
    e_off = 0
    crossings = 0
    for i, x in enumerate(ins):
        info, d, p = _sim(pic, x["nodes"], x["tris"], x["be"], x["bt"], dt, x["z"], x["r"],
                          x["ur"], x["up"], x["uz"], steps)
        crossings += d["n_crossings"]
        ne, nt = info["n_edges"], info["n_tris"]
        t0, t1 = u["tri_off"][i], u["tri_off"][i + 1]
        p0, p1 = u["part_off"][i], u["part_off"][i + 1]
        assert t1 - t0 == nt
        for k in ("E", "J"):
            a, b = du[k][e_off:e_off + ne], d[k]
            assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max(), (i, k)
        a, b = du["B"][t0:t1], d["B"]
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max(), (i, "B")
        # particles by id: union ids are the instance's shifted by the ones before it
        sel = (pu["pid"] >= p0) & (pu["pid"] < p1)
        assert np.array_equal(pu["pid"][sel] - p0, p["pid"])
        live = p["tri"] >= 0
        assert np.array_equal(pu["tri"][sel] >= 0, live)
        interior = live & (p["lam"].min(1) > 1e-5)
        assert np.array_equal(pu["tri"][sel][interior] - t0, p["tri"][interior])
        assert np.abs(pu["lam"][sel][live] - p["lam"][live]).max() < 1e-5
        assert np.abs(pu["u"][sel][live] - p["u"][live]).max() < 1e-5 * np.abs(p["u"]).max()
        e_off += ne
    assert e_off == info_u["n_edges"]
    assert crossings > 0 and abs(du["n_crossings"] - crossings) <= 1e-3 * crossings
    assert du["dce_nonzero"] == 0


def test_union_with_graph_replay_matches_the_oracle(pic):
    """The batched path as the sweep runs it -- the union of three instances as one
    simulation, each period of steps replayed as a CUDA graph -- against the FP64 oracle run on the same union mesh (coarse meshes, 1% of
    the particles).  20 steps from zero fields: per instance, E, B and J within 1e-5 of
    their largest magnitude (measured: below 1e-6), particle positions within 1e-5 of the mean edge length,
    momenta within 1e-5; triangle ids equal away from edges; continuity exact in
    integers."""
    from oracle import OracleSim
    ins = [sweep_instance(i, scale=0.01, mesh_scale=0.1) for i in range(3)]
    u = union(ins)
    o = OracleSim(u["nodes"], u["tris"], u["be"], u["bt"], eps0=EPS0, mu0=MU0, c=C0)
    dt = 0.5 * o.dt_max
    o.create(dt, bz=BZ_BWO)
    m = o.mesh
    o.set_fields(np.zeros(m.N1), np.zeros(m.N2))
    args = (u["z"], u["r"], u["ur"], u["up"], u["uz"], QE, ME, WEIGHT)
    o.inject(*args)
    mesh, dt_max = _mesh(pic, u["nodes"], u["tris"], u["be"], u["bt"])
    assert abs(dt_max - o.dt_max) <= 1e-6 * o.dt_max
    info = pic.pic_mesh_info(mesh)
    n = len(u["z"])
    sim = pic.pic_sim_create(mesh, dt, BZ_BWO, n + 1024)
    pic.pic_sim_set_sort_interval(sim, 4)
    pic.pic_sim_set_graph(sim, True)
    pic.pic_fields_set(sim, np.zeros(info["n_edges"]), np.zeros(info["n_tris"]))
    pic.pic_particles_inject(sim, *args)
    steps = 20
    pic.pic_step(sim, steps)
    o.step(steps)
    d = pic.pic_diagnostics(sim, fields=True)
    assert d["dce_nonzero"] == 0
    p = pic.pic_particles_get(sim)
    tri = -np.ones(n, np.int64)
    lam = np.zeros((n, 3))
    uu = np.zeros((n, 3))
    lv = p["tri"] >= 0
    tri[p["pid"][lv]] = p["tri"][lv]
    lam[p["pid"][lv]] = p["lam"][lv]
    uu[p["pid"][lv]] = p["u"][lv]
    live = o.tri >= 0
    assert np.array_equal(tri >= 0, live)
    assert d["n_crossings"] > 0 and abs(d["n_crossings"] - o.counters[2]) <= 1e-3 * o.counters[2]
    h = np.sqrt(2 * m.area.mean())
    xg = np.einsum("nk,nkd->nd", lam[live], u["nodes"][u["tris"][tri[live]]])
    xo = np.einsum("nk,nkd->nd", o.lam[live], u["nodes"][u["tris"][o.tri[live]]])
    err = {"pos": np.abs(xg - xo).max() / h,
           "u": np.abs(uu[live] - o.u[live]).max() / np.abs(o.u).max()}
    interior = live & (o.lam.min(1) > 1e-5)
    assert np.array_equal(tri[interior], o.tri[interior])
    # per instance: its edges, faces (triangles) in the union's numbering
    edge_inst = np.searchsorted(u["tri_off"], m.edge_tris[:, 0], side="right") - 1
    for i in range(len(ins)):
        t0, t1 = u["tri_off"][i], u["tri_off"][i + 1]
        e = edge_inst == i
        for k, a, b in (("E", d["E"][e], o.E[e]), ("J", d["J"][e], o.J[e]),
                        ("B", d["B"][t0:t1], o.B[t0:t1])):
            err["%s%d" % (k, i)] = np.abs(a - b).max() / np.abs(b).max()
    print(err)
    assert err["pos"] < 1e-5 and err["u"] < 1e-5
    for k, v in err.items():
        if k[0] in "EJB":
            assert v < 1e-5, (k, v)
