"""Sources on the GPU (Secs. 5.2, 5.3): the static gun field at the gather and cathode
emission against the oracle step by step, emission under graph replay and re-sorting,
the emitter's capacity rule, and a planar diode settling to the space-charge-limited
current."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import OracleSim, sources as S
from oracle import particles as OP

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
def cavity():
    arrays = W.cavity_mesh()
    return arrays, OracleSim(*arrays)


def _fresh(o):
    s = OracleSim.__new__(OracleSim)
    s.__dict__.update({k: (v.copy() if isinstance(v, np.ndarray) else v)
                       for k, v in o.__dict__.items()})
    return s


EMIT = dict(z0=0.013, rho0=0.0, rho1=0.35, u_normal=0.3, u_thermal=0.05, seed=11)


def _pair(pic, cavity, prec, n0, per_step, static):
    arrays, oracle = cavity
    nodes, tris, be, bt = arrays
    o = _fresh(oracle)
    m = o.mesh
    dt = 0.5 * o.dt_max
    o.create(dt, bz=0.3)
    E0 = W.random_edge_values(m.N1, 0.02, 40)
    o.set_fields(E0, np.zeros(m.N2))
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, precision=prec)
    pic.pic_spai_build(mesh)
    sim = pic.pic_sim_create(mesh, dt, 0.3, 200_000)
    pic.pic_sim_set_sort_interval(sim, 3)
    pic.pic_fields_set(sim, E0, np.zeros(m.N2))
    if n0:
        z, r, ur, up, uz = W.uniform_in_mesh(nodes, m.tris, n0, 41, sigma_u=0.3)
        o.inject(z, r, ur, up, uz, -1.0, 1.0, 1e-3)
        pic.pic_particles_inject(sim, z, r, ur, up, uz, -1.0, 1.0, 1e-3)
    if static:
        held = np.flatnonzero((m.nodes[:, 0] == 0.0) | (m.nodes[:, 0] == 1.0))
        _, Es = S.static_potential(m, o.star_eps, held, np.where(m.nodes[held, 0] == 0.0, 0.0, 0.5))
        o.set_static_field(Es)
        pic.pic_sim_set_static_field(sim, Es)
    if per_step:
        e = EMIT
        o.set_emitter(e["z0"], e["rho0"], e["rho1"], per_step, e["u_normal"], e["u_thermal"],
                      e["seed"], -1.0, 1.0, 1e-3)
        pic.pic_sim_set_emitter(sim, e["z0"], e["rho0"], e["rho1"], per_step, e["u_normal"],
                                e["u_thermal"], e["seed"], -1.0, 1.0, 1e-3)
    return o, sim, mesh


def _by_pid(pic, sim, n):
    p = pic.pic_particles_get(sim)
    tri = -np.ones(n, np.int64)
    lam = np.zeros((n, 3))
    u = np.zeros((n, 3))
    live = p["tri"] >= 0
    assert p["pid"][live].max() < n
    tri[p["pid"][live]] = p["tri"][live]
    lam[p["pid"][live]] = p["lam"][live]
    u[p["pid"][live]] = p["u"][live]
    return tri, lam, u


def _positions(nodes, tris, tri, lam):
    p = nodes[tris[np.maximum(tri, 0)]]
    return np.einsum("nk,nkd->nd", lam, p)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n0,per_step,static", [(3000, 0, True), (0, 400, False),
                                                (2000, 300, True)])
def test_sources_match_oracle(pic, cavity, prec, n0, per_step, static):
    """4 steps: particles, fields, currents and charges against the oracle (FP64: 1e-12;
    FP32: 1e-5 as in the step parity tests), DCE exact in the FP32 build, Gauss-law
    drift at round-off with the births taken out."""
    P = pic.PIC_FP64 if prec == "fp64" else pic.PIC_FP32
    o, sim, mesh = _pair(pic, cavity, P, n0, per_step, static)
    steps = 4
    pic.pic_step(sim, steps)
    for _ in range(steps):
        o.step()
    n = len(o.tri)
    assert n == n0 + steps * per_step
    d = pic.pic_diagnostics(sim, fields=True)
    assert d["n_emitted"] == steps * per_step and d["emit_dropped"] == 0
    tri, lam, u = _by_pid(pic, sim, n)
    live = o.tri >= 0
    assert np.array_equal(tri >= 0, live)
    nodes = cavity[0][0]
    xg = _positions(nodes, o.mesh.tris, tri, lam)
    xo = _positions(nodes, o.mesh.tris, o.tri, o.lam)
    tol = 1e-12 * steps if prec == "fp64" else 1e-5
    h = math.sqrt(2 * o.mesh.area.mean())
    assert np.abs(xg[live] - xo[live]).max() < tol * h
    assert np.abs(u[live] - o.u[live]).max() < tol * np.abs(o.u).max()
    for k, ref in (("E", o.E), ("B", o.B), ("J", o.J)):
        assert np.abs(d[k] - ref).max() <= tol * np.abs(ref).max(), k
    Q, Qp, Qa = pic.pic_charges_get(sim)
    assert np.abs(Q - o.Q).max() <= tol * np.abs(o.Q).max()
    if prec == "fp32":
        assert d["dce_nonzero"] == 0
    else:
        assert d["dce_max"] < 1e-12
    assert d["dgl_drift"] < (1e-12 if prec == "fp64" else 1e-5)


def test_emission_under_graph_replay_is_plain_steps(pic, cavity):
    """FP32: 30 steps with 500 births a step and a re-sort every 3 steps, in calls of 1, 7
    and 22 steps with and without graph replay: bit-identical states."""
    runs = []
    for graph in (False, True):
        o, sim, mesh = _pair(pic, cavity, pic.PIC_FP32, 1000, 500, True)
        pic.pic_sim_set_graph(sim, graph)
        for k in (1, 7, 22):
            pic.pic_step(sim, k)
        d = pic.pic_diagnostics(sim, fields=True)
        g = pic.pic_particles_get(sim)
        order = np.argsort(g["pid"])
        runs.append(({k: g[k][order] for k in ("pid", "tri", "lam", "u")}, d))
    (g1, d1), (g2, d2) = runs
    assert d1["n_emitted"] == d2["n_emitted"] == 30 * 500
    for k in ("pid", "tri", "lam", "u"):
        assert np.array_equal(g1[k], g2[k]), k
    for k in ("E", "B", "J", "n_absorbed", "dce_nonzero"):
        assert np.array_equal(d1[k], d2[k]), k


def test_emitter_capacity_and_arguments(pic, cavity):
    arrays, oracle = cavity
    nodes, tris, be, bt = arrays
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, precision=pic.PIC_FP32)
    dt = pic.pic_spai_build(mesh)
    sim = pic.pic_sim_create(mesh, 0.5 * dt, 0.0, 1000)
    pic.pic_sim_set_sort_interval(sim, 0)
    pic.pic_sim_set_emitter(sim, 0.013, 0.0, 0.35, 300, 0.0, 0.0, 3, -1.0, 1.0, 1e-3)
    pic.pic_step(sim, 5)       # 3 x 300 fit in 1000 slots, then two steps make none
    d = pic.pic_diagnostics(sim)
    assert d["n_emitted"] == 900 and d["emit_dropped"] == 600
    assert pic.pic_particles_count(sim) == 900
    for bad in (dict(z=-1.0), dict(rho1=-0.1), dict(q=1.0)):
        a = dict(z=0.013, rho0=0.0, rho1=0.35, per_step=10, u_normal=0.0, u_thermal=0.0,
                 seed=1, q=-1.0, m=1.0, w=1e-3)
        a.update(bad)
        with pytest.raises(pic.PicError) as e:
            pic.pic_sim_set_emitter(sim, **a)
        assert e.value.status == pic.PIC_ERR_ARG
    pic.pic_sim_set_emitter(sim, None, 0, 0, None, 0, 0, 0, 0, 0, 0)
    pic.pic_step(sim, 1)
    assert pic.pic_diagnostics(sim)["n_emitted"] == 900


def test_planar_diode_space_charge_limit(pic):
    """Sec. 5.2's diode check on a planar gap: 100 kV across 1 cm, emission at rest from a
    6 cm disk in a 7 cm tube, about 20k triangles graded toward the cathode, 2000 births
    per step, a 5 T guide field (one-dimensional flow), 10,000 settling and 10,000
    measured steps.  Injecting 0.95 of the relativistic planar space-charge-limited
    current, no particle returns to the cathode, the anode collects what is emitted and
    the central current density is the injected one; injecting 1.3 of it, a virtual
    cathode sends the excess back and the central current density that crosses the gap
    is the space-charge-limited one within 5%."""
    from paper_1701_03784_gb300 import diode
    from workloads.bwo import EPS0, C0, QE, ME
    J_scl = S.child_langmuir_planar(1e5, 1e-2, QE / ME, EPS0, C0)
    J_cl = diode.classical_limit(1e5, 1e-2)
    below = diode.run(over=0.95 * J_scl / J_cl)
    assert below["return_fraction"] == 0.0 and below["emit_dropped"] == 0
    assert below["dce_nonzero"] == 0
    assert below["n_emitted"] == below["n_particles"] + below["n_absorbed"]
    assert abs(below["I_anode"] / below["I_emitted"] - 1.0) < 0.01
    assert abs(below["J_center"] / J_scl - 0.95) < 0.05
    above = diode.run(over=1.3 * J_scl / J_cl)
    assert above["emit_dropped"] == 0 and above["dce_nonzero"] == 0
    assert above["return_fraction"] > 0.1
    assert abs(above["J_center"] / J_scl - 1.0) < 0.05, above["J_center"] / J_scl
