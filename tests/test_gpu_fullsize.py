"""Parity at the benchmark's full size and launch configuration: the single-BWO workload
with 16M particles, FP32 build, re-sort every 16 steps.  The oracle cannot push 16M
particles in seconds, so it pushes a random sample of them one by one from the same
state and fields; what must hold at any size is checked on the whole state (the
fixed-point continuity equation, Eq. charge recomputed from the positions, total charge)."""
import math

import numpy as np
import pytest

from workloads.bwo import bwo_workload, bwo_edge_field, EPS0, MU0, C0, QE, ME

pytestmark = pytest.mark.gpu

N_FULL = 16_000_000
N_SAMPLE = 20_000


@pytest.fixture(scope="module")
def pic():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import pic as p
    return p


def test_full_size_sampled_parity(pic):
    from oracle.operators import Mesh
    from oracle import particles as OP

    wl = bwo_workload(N_FULL)
    mesh = pic.pic_mesh_create(wl["nodes"], wl["tris"], wl["be"], wl["bt"], eps0=EPS0, mu0=MU0,
                               c=C0, precision=pic.PIC_FP32)
    pic.pic_spai_build(mesh, 2, 1e-4)
    info = pic.pic_mesh_info(mesh)
    sim = pic.pic_sim_create(mesh, wl["dt"], wl["bz"], N_FULL + 1024)
    pic.pic_sim_set_sort_interval(sim, 16)
    E0 = bwo_edge_field(info["n_edges"], wl["e_scale"], 7)
    pic.pic_fields_set(sim, E0, np.zeros(info["n_tris"]))
    pic.pic_particles_inject(sim, wl["z"], wl["r"], wl["ur"], wl["up"], wl["uz"], QE, ME,
                             wl["weight"])
    q0 = pic.pic_charges_get(sim)[0].sum()
    pic.pic_step(sim, 1)
    d = pic.pic_diagnostics(sim)
    # exact in the fixed-point build, at full size
    assert d["dce_nonzero"] == 0 and d["walk_overflows"] == 0
    Q, Qp, Qa = pic.pic_charges_get(sim)
    assert abs(Q.sum() + Qa.sum() - q0) <= 1e-12 * abs(q0)
    assert d["n_particles"] + d["n_absorbed"] == N_FULL

    # oracle: the same step for a sample of the particles, from the same input state
    p = pic.pic_particles_get(sim)
    order = np.argsort(p["pid"])
    rng = np.random.default_rng(5)
    sample = np.sort(rng.choice(N_FULL, N_SAMPLE, replace=False))
    m = Mesh(wl["nodes"], wl["tris"], wl["be"], wl["bt"])
    pm = OP.PushMesh(m)
    E = E0.copy()
    E[m.edge_tag == 1] = 0.0
    B_half = -wl["dt"] * (m.Dcurl @ E)          # B^{-1/2} = 0
    tri, lam = OP.locate(m, wl["z"][sample], wl["r"][sample])
    tri = np.ascontiguousarray(tri)
    lam = np.ascontiguousarray(lam)
    u = np.ascontiguousarray(np.stack([wl["ur"][sample], wl["up"][sample], wl["uz"][sample]], 1))
    J, Qs, Qas = np.zeros(m.N1), np.zeros(m.N0), np.zeros(m.N0)
    OP.push(pm, E, 0.5 * B_half, wl["bz"], wl["dt"], QE / ME, C0,
            wl["weight"] * QE / (2 * math.pi), tri, lam, u, J, Qs, Qas)

    g_tri = p["tri"][order][sample]
    g_lam = p["lam"][order][sample]
    g_u = p["u"][order][sample]
    live = tri >= 0
    assert np.array_equal(g_tri >= 0, live)
    h = math.sqrt(2 * m.area.mean())
    pos = lambda t, l: np.einsum("nk,nkd->nd", l, m.nodes[m.tris[np.maximum(t, 0)]])
    assert np.abs(pos(g_tri, g_lam)[live] - pos(tri, lam)[live]).max() < 1e-5 * h
    interior = live & (lam.min(1) > 1e-5)
    assert np.array_equal(g_tri[interior], tri[interior])
    assert np.abs(g_u[live] - u[live]).max() < 1e-5 * np.abs(u).max()
    # the sample really exercised the walk
    assert np.count_nonzero(g_tri[live] != OP.locate(m, wl["z"][sample], wl["r"][sample])[0][live]) > 100


def test_runs_are_bit_identical(pic):
    """Two simulations from the same inputs end in the same state, bit for bit, after 40
    steps (two re-sorts) on the BWO mesh with 2M particles: the fixed-point sums do not
    depend on the order of the atomics, and a particle's walk does not depend on which
    warp or ring pass handles it.  Compared per particle id (a re-sort may order the
    particles of one triangle differently)."""
    wl = bwo_workload(2_000_000)
    mesh = pic.pic_mesh_create(wl["nodes"], wl["tris"], wl["be"], wl["bt"], eps0=EPS0, mu0=MU0,
                               c=C0, precision=pic.PIC_FP32)
    pic.pic_spai_build(mesh, 2, 1e-4)
    info = pic.pic_mesh_info(mesh)
    E0 = bwo_edge_field(info["n_edges"], wl["e_scale"], 7)
    runs = []
    for _ in range(2):
        sim = pic.pic_sim_create(mesh, wl["dt"], wl["bz"], 2_000_000 + 1024)
        pic.pic_sim_set_sort_interval(sim, 16)
        pic.pic_fields_set(sim, E0, np.zeros(info["n_tris"]))
        pic.pic_particles_inject(sim, wl["z"], wl["r"], wl["ur"], wl["up"], wl["uz"], QE, ME,
                                 wl["weight"])
        pic.pic_step(sim, 40)
        d = pic.pic_diagnostics(sim, fields=True)
        p = pic.pic_particles_get(sim)
        order = np.argsort(p["pid"])
        runs.append(({k: p[k][order] for k in ("tri", "lam", "u", "pid")}, d,
                     pic.pic_charges_get(sim)))
        pic.pic_sim_destroy(sim)
    (p1, d1, q1), (p2, d2, q2) = runs
    assert d1["n_crossings"] > 10_000_000
    for k in ("tri", "lam", "u", "pid"):
        assert np.array_equal(p1[k], p2[k]), k
    for k in ("E", "B", "J", "n_crossings", "n_absorbed", "dce_nonzero"):
        assert np.array_equal(d1[k], d2[k]), k
    for a, b in zip(q1, q2):
        assert np.array_equal(a, b)
