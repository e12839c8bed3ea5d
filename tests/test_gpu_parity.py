"""GPU parity: the CUDA path, called through the C ABI, against the FP64 oracle on the same
seeded inputs.  FP64 build: 1e-12 relative per step.  FP32 build (fixed-point positions
and currents): 1e-5 relative per step, and the discrete continuity equation exact in
integers."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import OracleSim
from oracle.operators import Mesh
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
def cavity_oracle():
    nodes, tris, be, bt = W.cavity_mesh()          # 0.5 x 1 cavity, ~2000 triangles
    return (nodes, tris, be, bt), OracleSim(nodes, tris, be, bt)


def _copy(o):
    """A fresh oracle state sharing only the read-only operators of a prepared one."""
    s = OracleSim.__new__(OracleSim)
    s.__dict__.update({k: (v.copy() if isinstance(v, np.ndarray) else v)
                       for k, v in o.__dict__.items()})
    m = s.mesh
    s.Q, s.Q_prev, s.Qabs = np.zeros(m.N0), np.zeros(m.N0), np.zeros(m.N0)
    s.J = np.zeros(m.N1)
    s.counters = np.zeros(3, np.int64)
    return s


def _setup(pic, mesh_arrays, oracle, prec, n, seed, dt_frac=0.5, bz=0.3, sigma_u=0.3,
           e_scale=0.05, walk_cap=0, sort_interval=4, cap=None, pusher="boris"):
    nodes, tris, be, bt = mesh_arrays
    o = _copy(oracle)
    m = o.mesh
    dt = dt_frac * o.dt_max
    o.create(dt, bz=bz)
    E0 = W.random_edge_values(m.N1, e_scale, seed)
    B0 = W.random_edge_values(m.N2, 1e-3, seed + 1)
    o.set_fields(E0, B0)
    z, r, ur, up, uz = W.uniform_in_mesh(nodes, tris, n, seed + 2, sigma_u=sigma_u)
    o.inject(z, r, ur, up, uz, -1.0, 1.0, 1e-3)
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, precision=prec, walk_cap=walk_cap)
    pic.pic_spai_build(mesh)
    sim = pic.pic_sim_create(mesh, dt, bz, cap or 2 * n + 16)
    pic.pic_sim_set_sort_interval(sim, sort_interval)
    if pusher == "vay":
        o.pusher = OP.VAY
        pic.pic_sim_set_pusher(sim, pic.PIC_PUSHER_VAY)
    pic.pic_fields_set(sim, E0, B0)
    pic.pic_particles_inject(sim, z, r, ur, up, uz, -1.0, 1.0, 1e-3)
    if walk_cap:
        o_cap = walk_cap
    else:
        o_cap = OP.WALK_CAP
    return o, sim, mesh, o_cap


def _gpu_particles(pic, sim, n):
    p = pic.pic_particles_get(sim)
    tri = -np.ones(n, np.int64)
    lam = np.zeros((n, 3))
    u = np.zeros((n, 3))
    live = p["tri"] >= 0
    tri[p["pid"][live]] = p["tri"][live]
    lam[p["pid"][live]] = p["lam"][live]
    u[p["pid"][live]] = p["u"][live]
    return tri, lam, u


def _oracle_step(o, n_steps, cap):
    for _ in range(n_steps):
        B_half = o.field_b_half()
        m = o.mesh
        Bavg = 0.5 * (B_half + o.B)
        o.J = np.zeros(m.N1)
        Qn = np.zeros(m.N0)
        o.Qabs = np.zeros(m.N0)
        o.counters += OP.push(o.pm, o.E, Bavg, o.bz, o.dt, o.qm, o.c, o.q_src, o.tri, o.lam,
                              o.u, o.J, Qn, o.Qabs, max_cross=cap, pusher=o.pusher)
        o.field_e(B_half)
        o.B = B_half
        o.Q_prev, o.Q = o.Q, Qn


def _elementwise(a, ref, floor, rtol):
    """Per-element relative agreement where the reference is not tiny: every entry with
    |ref| >= floor * max|ref| is within rtol of it (the normwise checks bound the rest)."""
    big = np.abs(ref) >= floor * np.abs(ref).max()
    assert big.sum() > 0
    err = np.abs(a[big] - ref[big]) / np.abs(ref[big])
    assert err.max() <= rtol, (err.max(), int(big.sum()))


def _positions(nodes, tris, tri, lam):
    p = nodes[tris[np.maximum(tri, 0)]]
    return np.einsum("nk,nkd->nd", lam, p)


@pytest.mark.parametrize("pusher", ["boris", "vay"])
@pytest.mark.parametrize("steps", [1, 5])
def test_fp64_matches_oracle(pic, cavity_oracle, steps, pusher):
    """FP64 build: particle state, fields and scatter within 1e-12 of the oracle."""
    arrays, oracle = cavity_oracle
    n = 10_000
    o, sim, mesh, cap = _setup(pic, arrays, oracle, pic.PIC_FP64, n, seed=10, pusher=pusher)
    pic.pic_step(sim, steps)
    _oracle_step(o, steps, cap)
    d = pic.pic_diagnostics(sim, fields=True)
    tri, lam, u = _gpu_particles(pic, sim, n)
    assert np.array_equal(tri, o.tri)
    live = o.tri >= 0
    tol = 1e-12 * steps
    assert np.abs(lam[live] - o.lam[live]).max() < tol
    assert np.abs(u[live] - o.u[live]).max() < tol * np.abs(o.u).max()
    assert np.abs(d["E"] - o.E).max() < tol * np.abs(o.E).max()
    assert np.abs(d["B"] - o.B).max() < tol * np.abs(o.B).max()
    assert np.abs(d["J"] - o.J).max() < tol * np.abs(o.J).max()
    Q, Qp, Qa = pic.pic_charges_get(sim)
    assert np.abs(Q - o.Q).max() < tol * np.abs(o.Q).max()
    assert np.abs(Qa - o.Qabs).max() < tol * max(np.abs(o.Q).max(), 1e-30)
    # per element: edges and nodes down to 1e-6 of the largest value, 1e-9 relative
    _elementwise(d["J"], o.J, 1e-6, 1e-9)
    _elementwise(Q, o.Q, 1e-6, 1e-9)
    assert d["n_absorbed"] == o.counters[0] and d["n_crossings"] == o.counters[2]
    assert d["dce_max"] < 1e-12 and d["dgl_drift"] < 1e-12


@pytest.mark.parametrize("pusher", ["boris", "vay"])
@pytest.mark.parametrize("steps", [1, 3])
def test_fp32_matches_oracle(pic, cavity_oracle, steps, pusher):
    """FP32 build: 1e-5 relative per step; triangle ids equal except within 1e-5 of an edge."""
    arrays, oracle = cavity_oracle
    nodes, tris = arrays[0], arrays[1]
    n = 10_000
    o, sim, mesh, cap = _setup(pic, arrays, oracle, pic.PIC_FP32, n, seed=20, pusher=pusher)
    pic.pic_step(sim, steps)
    _oracle_step(o, steps, cap)
    d = pic.pic_diagnostics(sim, fields=True)
    tri, lam, u = _gpu_particles(pic, sim, n)
    tol = 1e-5
    live = o.tri >= 0
    assert np.array_equal(tri >= 0, live)
    h = math.sqrt(2 * o.mesh.area.mean())
    xg = _positions(nodes, o.mesh.tris, tri, lam)
    xo = _positions(nodes, o.mesh.tris, o.tri, o.lam)
    assert np.abs(xg[live] - xo[live]).max() < tol * h
    interior = live & (o.lam.min(1) > 1e-5)
    assert np.array_equal(tri[interior], o.tri[interior])
    assert np.abs(u[live] - o.u[live]).max() < tol * np.abs(o.u).max()
    assert np.abs(d["E"] - o.E).max() < tol * np.abs(o.E).max()
    assert np.abs(d["B"] - o.B).max() < tol * np.abs(o.B).max()
    assert np.abs(d["J"] - o.J).max() < tol * np.abs(o.J).max()
    # charge conservation is exact in the fixed-point build
    assert d["dce_nonzero"] == 0 and d["dce_max"] == 0.0
    Q, Qp, Qa = pic.pic_charges_get(sim)
    assert np.abs(Q - o.Q).max() < tol * np.abs(o.Q).max()
    # per element: edges and nodes down to 1% of the largest value within 1e-3 relative
    # (the fixed-point positions round at 2^-22 of a cell, so an entry's error does not
    # shrink with its size; below 1% of the maximum the normwise bound above applies)
    _elementwise(d["J"], o.J, 1e-2, 1e-3)
    _elementwise(Q, o.Q, 1e-2, 1e-3)


def test_fp32_dce_exact_over_many_steps(pic, cavity_oracle):
    """50 steps with re-sorting every 3 steps: the fixed-point DCE residual is exactly zero
    at every step, the DGL residual stays constant, and total charge is conserved."""
    arrays, oracle = cavity_oracle
    o, sim, mesh, cap = _setup(pic, arrays, oracle, pic.PIC_FP32, 20_000, seed=30,
                               sigma_u=0.8, sort_interval=3)
    q0 = pic.pic_charges_get(sim)[0].sum()
    qabs = 0.0
    for k in range(50):
        pic.pic_step(sim, 1)
        d = pic.pic_diagnostics(sim)
        assert d["dce_nonzero"] == 0, k
        Q, Qp, Qa = pic.pic_charges_get(sim)
        qabs += Qa.sum()
        assert abs(Q.sum() + qabs - q0) <= 1e-12 * abs(q0)
    assert d["dgl_drift"] < 1e-5
    assert d["n_absorbed"] > 0 and d["n_crossings"] > 0


def test_walk_cap_and_empty(pic, cavity_oracle):
    """walk_cap = 1 removes a particle at its second crossing, as in the oracle; a
    simulation without particles steps its fields like the oracle."""
    arrays, oracle = cavity_oracle
    n = 5000
    o, sim, mesh, cap = _setup(pic, arrays, oracle, pic.PIC_FP64, n, seed=40, sigma_u=3.0,
                               walk_cap=1)
    pic.pic_step(sim, 2)
    _oracle_step(o, 2, cap)
    d = pic.pic_diagnostics(sim)
    assert d["walk_overflows"] == o.counters[1] and d["n_absorbed"] == o.counters[0]
    tri, lam, u = _gpu_particles(pic, sim, n)
    assert np.array_equal(tri, o.tri)

    o2 = _copy(oracle)
    o2.create(0.5 * o2.dt_max)
    m = o2.mesh
    E0 = W.tm0np_edge_dofs(m.nodes, m.edge_nodes, 0.5, 1.0, 1, 1)
    o2.set_fields(E0, np.zeros(m.N2))
    mesh2 = pic.pic_mesh_create(*arrays, precision=pic.PIC_FP64)
    pic.pic_spai_build(mesh2)
    sim2 = pic.pic_sim_create(mesh2, o2.dt, 0.0, 0)
    pic.pic_fields_set(sim2, E0, np.zeros(m.N2))
    pic.pic_step(sim2, 20)
    o2.step(20)
    d2 = pic.pic_diagnostics(sim2, fields=True)
    assert np.abs(d2["E"] - o2.E).max() < 1e-12 * np.abs(o2.E).max()
    assert d2["n_particles"] == 0


def test_rest_particles_are_bit_exact(pic, cavity_oracle):
    """Particles at rest in zero fields keep their fixed-point coordinates bit for bit and
    deposit no current."""
    arrays, oracle = cavity_oracle
    nodes, tris, be, bt = arrays
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, precision=pic.PIC_FP32)
    dt = 0.5 * pic.pic_spai_build(mesh)
    sim = pic.pic_sim_create(mesh, dt, 0.0, 1000)
    z, r, *_ = W.uniform_in_mesh(nodes, tris, 500, 7)
    zero = np.zeros(500)
    pic.pic_particles_inject(sim, z, r, zero, zero, zero, -1.0, 1.0, 1e-3)
    p0 = pic.pic_particles_get(sim)
    pic.pic_step(sim, 3)
    p1 = pic.pic_particles_get(sim)
    o0, o1 = np.argsort(p0["pid"]), np.argsort(p1["pid"])
    assert np.array_equal(p0["tri"][o0], p1["tri"][o1])
    assert np.array_equal(p0["lam"][o0], p1["lam"][o1])
    d = pic.pic_diagnostics(sim, fields=True)
    assert np.all(d["J"] == 0) and np.all(d["E"] == 0)


def test_resort_orders_by_triangle(pic, cavity_oracle):
    arrays, oracle = cavity_oracle
    o, sim, mesh, cap = _setup(pic, arrays, oracle, pic.PIC_FP32, 30_000, seed=50, sigma_u=1.0,
                               sort_interval=2)
    pic.pic_step(sim, 4)
    p = pic.pic_particles_get(sim)
    assert np.all(np.diff(p["tri"]) >= 0) and p["tri"][0] >= 0
    d = pic.pic_diagnostics(sim)
    assert len(p["pid"]) == d["n_particles"]
    assert len(np.unique(p["pid"])) == len(p["pid"])


def test_raw_roundtrip(pic, cavity_oracle):
    """Host round trip of the raw state leaves the simulation unchanged."""
    import torch
    arrays, oracle = cavity_oracle
    o, sim, mesh, cap = _setup(pic, arrays, oracle, pic.PIC_FP32, 4000, seed=60)
    n = pic.pic_particles_count(sim)
    b = pic.pic_particles_raw_bytes(sim)
    assert b == 24
    # every array of the raw layout starts on a 128-byte boundary
    for m in (0, 1, 31, 32, 33, n):
        assert pic.pic_particles_raw_size(sim, m) == -(-m // 32) * 32 * b
    buf = torch.empty(pic.pic_particles_raw_size(sim, n), dtype=torch.uint8, pin_memory=True)
    before = pic.pic_particles_get(sim)
    pic.pic_particles_raw_get(sim, buf.data_ptr(), n)
    torch.cuda.synchronize()
    pic.pic_particles_raw_set(sim, buf.data_ptr(), n)
    torch.cuda.synchronize()
    after = pic.pic_particles_get(sim)
    for k in ("tri", "lam", "u"):
        assert np.array_equal(before[k], after[k])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_dgl_holds_with_charge_leaving_at_open_ends(pic, prec):
    """Two-period BWO-shaped mesh with absorbing (non-conducting) ends, thermal particles
    that leave through them: the charge removed there leaves Q without crossing an edge,
    and once that is accounted for the Gauss-law residual D_div D - Q stays at round-off
    (Eq. DGL_RSD_REL)."""
    nodes, tris, be, bt = W.bwo_small_mesh(n_tri=3000, seed=4)
    p = pic.PIC_FP64 if prec == "fp64" else pic.PIC_FP32
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, precision=p)
    dt_max = pic.pic_spai_build(mesh)
    info = pic.pic_mesh_info(mesh)
    n = 20_000
    sim = pic.pic_sim_create(mesh, 0.5 * dt_max, 0.1, n + 16)
    pic.pic_sim_set_sort_interval(sim, 4)
    pic.pic_fields_set(sim, W.random_edge_values(info["n_edges"], 1e-3, 50),
                       np.zeros(info["n_tris"]))
    z, r, ur, up, uz = W.uniform_in_mesh(nodes, tris, n, 51, sigma_u=0.8)
    pic.pic_particles_inject(sim, z, r, ur, up, uz, -1.0, 1.0, 1e-3)
    on_pec = Mesh(nodes, tris, be, bt).node_on_pec.astype(bool)
    q_open = 0.0
    for _ in range(60):
        pic.pic_step(sim, 1)
        q_open += np.abs(pic.pic_charges_get(sim)[2][~on_pec]).sum()
    d = pic.pic_diagnostics(sim)
    assert q_open > 0 and d["n_absorbed"] > 0        # charge left through the open ends
    assert d["dgl_drift"] < (1e-10 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_step_host_matches_device_steps(pic, cavity_oracle, prec):
    """pic_step_host (the state uploaded from page-locked host memory, stepped and written
    back every step, with the two copy directions overlapped) ends in the same state, bit
    for bit, as the same steps on the device, and its host buffer holds that state.  Seven
    steps with re-sorts every 3 and particles leaving through the walls."""
    torch = pytest.importorskip("torch")
    arrays, oracle = cavity_oracle
    p = pic.PIC_FP64 if prec == "fp64" else pic.PIC_FP32
    n = 20_000
    runs = []
    for mode in ("device", "host"):
        o, sim, mesh, cap = _setup(pic, arrays, oracle, p, n, seed=60, sigma_u=0.8,
                                   sort_interval=3)
        nslot = pic.pic_particles_count(sim)
        bpp = pic.pic_particles_raw_bytes(sim)
        host = torch.empty(pic.pic_particles_raw_size(sim, nslot), dtype=torch.uint8,
                           pin_memory=True)
        pic.pic_particles_raw_get(sim, host.data_ptr(), nslot)
        torch.cuda.synchronize()
        if mode == "device":
            pic.pic_step(sim, 7)
        else:
            pic.pic_step_host(sim, host.data_ptr(), nslot, 7)
        torch.cuda.synchronize()
        d = pic.pic_diagnostics(sim, fields=True)
        g = pic.pic_particles_get(sim)
        order = np.argsort(g["pid"])
        if mode == "host":
            live = pic.pic_particles_count(sim)
            back = torch.empty(pic.pic_particles_raw_size(sim, nslot), dtype=torch.uint8,
                               pin_memory=True)
            pic.pic_particles_raw_get(sim, back.data_ptr(), live)
            torch.cuda.synchronize()
            # per array: the first `live` slots of the returned buffer are the device state
            # (array strides: the slot counts rounded up to 32)
            sizes = [4] + [(bpp - 4) // 5] * 5       # tri, then 5 arrays of one type
            hb, bb = host.numpy(), back.numpy()
            off_h = off_b = 0
            for sz in sizes:
                assert np.array_equal(hb[off_h:off_h + sz * live], bb[off_b:off_b + sz * live])
                off_h += sz * (-(-nslot // 32) * 32)
                off_b += sz * (-(-live // 32) * 32)
        runs.append(({k: g[k][order] for k in ("pid", "tri", "lam", "u")}, d))
    (g1, d1), (g2, d2) = runs
    assert d1["n_absorbed"] > 0 and d1["n_absorbed"] == d2["n_absorbed"]
    assert np.array_equal(g1["pid"], g2["pid"]) and np.array_equal(g1["tri"], g2["tri"])
    if prec == "fp32":
        # integer sums: bit for bit
        for k in ("lam", "u"):
            assert np.array_equal(g1[k], g2[k]), k
        for k in ("E", "B", "J"):
            assert np.array_equal(d1[k], d2[k]), k
    else:
        # the FP64 build sums with floating-point atomics, whose order varies: round-off
        for a, b in [(g1["lam"], g2["lam"]), (g1["u"], g2["u"])] + [(d1[k], d2[k]) for k in "EBJ"]:
            assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


def test_graph_replay_matches_plain_steps(pic, cavity_oracle):
    """pic_step replaying a CUDA graph of one period (re-sort every 3 steps: 6 steps) gives
    the state of plain steps, bit for bit in the FP32 build: 45 steps in calls of 1, 7, 13
    and 24 steps, so that periods start at different phases and tails run plainly; then 12
    more steps with the Vay pusher (the recorded graph must not be replayed for them)."""
    arrays, oracle = cavity_oracle
    runs = []
    for graph in (False, True):
        o, sim, mesh, cap = _setup(pic, arrays, oracle, pic.PIC_FP32, 20_000, seed=70,
                                   sigma_u=0.8, sort_interval=3)
        pic.pic_sim_set_graph(sim, graph)
        for k in (1, 7, 13, 24):
            pic.pic_step(sim, k)
        pic.pic_sim_set_pusher(sim, pic.PIC_PUSHER_VAY)
        pic.pic_step(sim, 12)
        d = pic.pic_diagnostics(sim, fields=True)
        g = pic.pic_particles_get(sim)
        order = np.argsort(g["pid"])
        runs.append(({k: g[k][order] for k in ("pid", "tri", "lam", "u")}, d))
    (g1, d1), (g2, d2) = runs
    assert d1["n_steps"] == d2["n_steps"] == 57 and d1["n_absorbed"] > 0
    for k in ("pid", "tri", "lam", "u"):
        assert np.array_equal(g1[k], g2[k]), k
    for k in ("E", "B", "J", "n_crossings", "n_absorbed", "dce_nonzero", "dgl_drift"):
        assert np.array_equal(d1[k], d2[k]), k


def test_autotune_changes_no_result(pic, cavity_oracle):
    """pic_sim_autotune tries re-sort intervals, particle-kernel grids and field-kernel block
    sizes while stepping: the FP32 state after it is bit for bit that of the same number
    of plain steps (14 trials of 8 steps)."""
    arrays, oracle = cavity_oracle
    runs = []
    for tune in (True, False):
        o, sim, mesh, cap = _setup(pic, arrays, oracle, pic.PIC_FP32, 20_000, seed=80,
                                   sigma_u=0.8, sort_interval=16)
        if tune:
            t = pic.pic_sim_autotune(sim, 8)
            assert t["sort_interval"] in (8, 16, 32) and t["ctas_per_sm"] in (0, 2, 3)
            assert t["field_block"] in (128, 256, 512) and t["ms_per_step"] > 0
        else:
            pic.pic_step(sim, 14 * 8)
        d = pic.pic_diagnostics(sim, fields=True)
        g = pic.pic_particles_get(sim)
        # removed particles keep their slots until a re-sort, and the runs re-sort at
        # different steps: compare the live ones
        live = np.nonzero(g["tri"] >= 0)[0]
        order = live[np.argsort(g["pid"][live])]
        runs.append(({k: g[k][order] for k in ("pid", "tri", "lam", "u")}, d))
    (g1, d1), (g2, d2) = runs
    assert d1["n_steps"] == d2["n_steps"] == 112
    for k in ("pid", "tri", "lam", "u"):
        assert np.array_equal(g1[k], g2[k]), k
    for k in ("E", "B", "J", "n_crossings", "n_absorbed", "dce_nonzero"):
        assert np.array_equal(d1[k], d2[k]), k


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_energy_diagnostics_match_the_oracle_definitions(pic, cavity_oracle, prec):
    """The device reductions behind pic_diagnostics: the kinetic energy (sum over live
    particles of (gamma - 1) m c^2 w) and the field energy (1/2 E star_eps E + 1/2 B
    star_mu^-1 B) equal the oracle's definitions evaluated on the state read back."""
    arrays, oracle = cavity_oracle
    P = pic.PIC_FP64 if prec == "fp64" else pic.PIC_FP32
    n = 30_000
    o, sim, mesh, cap = _setup(pic, arrays, oracle, P, n, seed=70, sigma_u=0.8)
    pic.pic_step(sim, 5)
    d = pic.pic_diagnostics(sim, fields=True)
    tri, lam, u = _gpu_particles(pic, sim, n)
    assert (tri >= 0).sum() == d["n_particles"]
    o.tri, o.u = tri, u
    o.E, o.B = d["E"], d["B"]
    # FP32 build: each (gamma - 1) term is evaluated in FP32, and the diagonal star_mu^-1
    # is stored in FP32 (relative rounding 6e-8 per face)
    tol = 1e-12 if prec == "fp64" else 2e-6
    assert d["kinetic_energy"] == pytest.approx(o.kinetic_energy(), rel=tol)
    assert d["field_energy"] == pytest.approx(o.field_energy(), rel=1e-12 if prec == "fp64" else 1e-7)
    # the plain read-back (no reductions) returns the same fields
    E, B = pic.pic_fields_get(sim)
    assert np.array_equal(E, d["E"]) and np.array_equal(B, d["B"])
    pic.pic_sim_destroy(sim)
    pic.pic_mesh_destroy(mesh)
