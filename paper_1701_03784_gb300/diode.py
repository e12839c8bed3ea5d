"""Planar space-charge-limited diode (the diode check of Sec. 5.2, on a planar gap): the
static field of the electrode voltage (pic_static_potential), emission at rest from a
cathode disk (pic_sim_set_emitter), and the current density that reaches the anode.

SI units.  Cathode plane z = 0 (potential 0), anode plane z = gap (potential V), outer
wall rho = radius; conducting walls everywhere but the axis.  Births at rest on the plane
z = emit_z * gap over rho < r_emit, `over` times the classical Child-Langmuir current.

Sec. 5.2 finds the limit as the largest injection that forms no virtual cathode; here a
virtual cathode shows as emitted particles returning to the cathode (`return_fraction`,
current to the cathode plane over the emitted current).  Below the limit the whole
emission reaches the anode; above it the excess returns and the current that crosses the
gap is the space-charge-limited one.  The defaults are the planar check: a 6 cm emitter
in a 7 cm tube (1 cm gap), so that the finite emitter's enhancement of the limit stays
at its edge; a 5 T guide field, so that the flow is one-dimensional (without it the
beam's own magnetic field, which the electrodes do not short out, pinches it toward the
axis); a mesh graded toward the cathode (`grade`), where the potential of the
space-charge-limited flow varies as z^(4/3).

Births sit 1e-6 gaps off the cathode.  A birth adds its charge to Q^n with no current,
so the field never sees the share of it that lands on nodes off the conductor (on
conductor nodes it is shorted out anyway): each birth at height z0 leaves about z0 / h
of its charge as a fixed charge of the opposite sign in the first row of nodes.  With
births 20 um off the cathode (0.2 of a cell) that sheet grew to a few kV of extra
extraction voltage over 20,000 steps and the transmitted current drifted upward; at 1e-6
gaps it stays below a few volts."""
import math

import numpy as np

from . import pic
from workloads.bwo import EPS0, MU0, C0, QE, ME
from workloads.meshes import diode_mesh


def classical_limit(V, gap):
    """Non-relativistic planar Child-Langmuir current density (A/m^2)."""
    return 4.0 * EPS0 / 9.0 * math.sqrt(2.0 * abs(QE) / ME) * V ** 1.5 / gap ** 2


def run(V=1e5, gap=1e-2, radius=7e-2, r_emit=6e-2, n_tri=20_000, per_step=2000, over=1.0,
        settle_steps=10_000, measure_steps=10_000, r_measure=1e-2, precision=pic.PIC_FP32,
        mesh_seed=1001, seed=77, graph=True, sort_interval=16, capacity=8_000_000,
        history_every=1000, bz=5.0, time_steps=0, emit_z=1e-6, grade=0.35):
    """Run the diode and return the anode current density within r_measure, averaged
    over measure_steps after settle_steps, with the run's figures (and the same density
    averaged over every history_every steps of the whole run, to show it settle)."""
    import torch
    nodes, tris, be, bt = diode_mesh(n_tri=n_tri, seed=mesh_seed, gap=gap, radius=radius,
                                     grade=grade)
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, eps0=EPS0, mu0=MU0, c=C0,
                               precision=precision)
    dt_max = pic.pic_spai_build(mesh, 2, 1e-4)
    dt = 0.5 * dt_max
    z = nodes[:, 0]
    held = np.flatnonzero((z == 0.0) | (z == gap))
    _, Es = pic.pic_static_potential(mesh, held, np.where(z[held] == 0.0, 0.0, V))
    sim = pic.pic_sim_create(mesh, dt, bz, capacity)
    pic.pic_sim_set_sort_interval(sim, sort_interval)
    pic.pic_sim_set_graph(sim, graph)
    pic.pic_sim_set_static_field(sim, Es)
    J_cl = classical_limit(V, gap)
    weight = over * J_cl * math.pi * r_emit ** 2 * dt / (per_step * abs(QE))
    pic.pic_sim_set_emitter(sim, emit_z * gap, 0.0, r_emit, per_step, 0.0, 0.0, seed, QE, ME,
                            weight)
    anode = np.flatnonzero(z == gap)
    anode = anode[np.argsort(nodes[anode, 1])]
    cathode = np.flatnonzero(z == 0.0)
    inside = anode[nodes[anode, 1] <= r_measure]
    rho_edge = 0.5 * (nodes[inside[-1], 1] + nodes[anode[len(inside)], 1])
    torch.cuda.synchronize()
    # node charges are per radian (the ring normalisation q w / (2 pi))
    area = math.pi * rho_edge ** 2
    history, hist_anode, hist_back, hist_live = [], [], [], []
    q_center = q_anode = q_win = q_back = qa_win = qb_win = 0.0
    total = settle_steps + measure_steps
    for k in range(total):
        pic.pic_step(sim, 1)
        _, _, Qa = pic.pic_charges_get(sim)
        qc = Qa[inside].sum()
        qa = Qa[anode].sum()
        qb = Qa[cathode].sum()
        q_win += qc
        qa_win += qa
        qb_win += qb
        if k >= settle_steps:
            q_center += qc
            q_anode += qa
            q_back += qb
        if (k + 1) % history_every == 0:
            w = history_every * dt
            history.append(abs(2.0 * math.pi * q_win) / w / area)
            hist_anode.append(abs(2.0 * math.pi * qa_win) / w)
            hist_back.append(abs(2.0 * math.pi * qb_win) / w)
            hist_live.append(pic.pic_diagnostics(sim)["n_particles"])
            q_win = qa_win = qb_win = 0.0
    d = pic.pic_diagnostics(sim)
    step_ms = None
    if time_steps:
        # throughput at the settled particle count: plain stepping, no read-back
        live = d["n_particles"]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pic.pic_step(sim, time_steps)
        e1.record()
        torch.cuda.synchronize()
        step_ms = e0.elapsed_time(e1) / time_steps
        live = 0.5 * (live + pic.pic_diagnostics(sim)["n_particles"])
    J = abs(2.0 * math.pi * q_center) / (measure_steps * dt) / area
    I_anode = abs(2.0 * math.pi * q_anode) / (measure_steps * dt)
    I_back = abs(2.0 * math.pi * q_back) / (measure_steps * dt)
    I_emit = over * J_cl * math.pi * r_emit ** 2
    out = {"J_center": J, "J_classical": J_cl, "rho_measure": rho_edge, "I_anode": I_anode,
           "I_emitted": I_emit, "I_returned": I_back, "return_fraction": I_back / I_emit,
           "dt": dt, "steps": d["n_steps"],
           "n_particles": d["n_particles"], "n_emitted": d["n_emitted"],
           "n_absorbed": d["n_absorbed"], "emit_dropped": d["emit_dropped"],
           "dce_nonzero": d["dce_nonzero"], "dgl_drift": d["dgl_drift"],
           "n_tris": len(tris), "J_center_history": history, "history_every": history_every,
           "I_anode_history": hist_anode, "I_returned_history": hist_back,
           "live_history": hist_live}
    if step_ms is not None:
        out.update(step_ms=step_ms, time_steps=time_steps,
                   particle_steps_per_s=live / (step_ms * 1e-3))
    pic.pic_sim_destroy(sim)
    pic.pic_mesh_destroy(mesh)
    return out


def throughput(V=1e5, gap=1e-2, radius=2e-2, r_emit=1e-2, n_tri=20_000, per_step=2000,
               over=1.0, settle_steps=4000, steps=1000, bz=0.0, emit_z=1e-6, grade=1.0,
               mesh_seed=1001, seed=77, sort_interval=16, capacity=8_000_000):
    """Steps per second of the diode once the gap has filled: settle_steps plain steps
    (graph replay, no read-back), then `steps` timed with CUDA events.  The defaults are the
    diode configuration as stated: a 1 cm cathode disk 1 cm from the anode in a 2 cm tube,
    about 20k triangles, 2000 births per step, FP32."""
    import torch
    nodes, tris, be, bt = diode_mesh(n_tri=n_tri, seed=mesh_seed, gap=gap, radius=radius,
                                     grade=grade)
    mesh = pic.pic_mesh_create(nodes, tris, be, bt, eps0=EPS0, mu0=MU0, c=C0,
                               precision=pic.PIC_FP32)
    dt = 0.5 * pic.pic_spai_build(mesh, 2, 1e-4)
    z = nodes[:, 0]
    held = np.flatnonzero((z == 0.0) | (z == gap))
    _, Es = pic.pic_static_potential(mesh, held, np.where(z[held] == 0.0, 0.0, V))
    sim = pic.pic_sim_create(mesh, dt, bz, capacity)
    pic.pic_sim_set_sort_interval(sim, sort_interval)
    pic.pic_sim_set_graph(sim, True)
    pic.pic_sim_set_static_field(sim, Es)
    weight = over * classical_limit(V, gap) * math.pi * r_emit ** 2 * dt / (per_step * abs(QE))
    pic.pic_sim_set_emitter(sim, emit_z * gap, 0.0, r_emit, per_step, 0.0, 0.0, seed, QE, ME,
                            weight)
    pic.pic_step(sim, settle_steps)
    torch.cuda.synchronize()
    live0 = pic.pic_diagnostics(sim)["n_particles"]
    pic.pic_kernel_timing(sim, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    pic.pic_step(sim, steps)
    e1.record()
    torch.cuda.synchronize()
    push_ms, n_push = pic.pic_kernel_timing(sim, False)
    d = pic.pic_diagnostics(sim)
    ms = e0.elapsed_time(e1) / steps
    live = 0.5 * (live0 + d["n_particles"])
    out = {"ms_per_step": ms, "push_ms": push_ms / max(n_push, 1), "steps": steps,
           "settle_steps": settle_steps, "in_flight": [live0, d["n_particles"]],
           "particle_steps_per_s": live / (ms * 1e-3), "dt": dt, "n_tris": len(tris),
           "births_per_step": per_step, "emit_dropped": d["emit_dropped"],
           "dce_nonzero": d["dce_nonzero"]}
    pic.pic_sim_destroy(sim)
    pic.pic_mesh_destroy(mesh)
    return out
