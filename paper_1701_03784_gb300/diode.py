"""Planar space-charge-limited diode (the diode check of Sec. 5.2, on a planar gap): the
static field of the electrode voltage (pic_static_potential), emission at rest from a
cathode disk at a current above what the gap can carry (pic_sim_set_emitter), and the
current density that reaches the anode once a virtual cathode has formed in front of the
emitter.  Away from the emitter's edge that is the one-dimensional space-charge-limited
current of the gap.

SI units.  Cathode plane z = 0 (potential 0), anode plane z = gap (potential V), outer
wall rho = radius; conducting walls everywhere but the axis.  Births at z = 2e-3 gap over
rho < r_emit, `over` times the classical Child-Langmuir current.  The emitter is wide
(6 cm against a 1 cm gap) so that the gap's space-charge limit is close to the planar one.

Sec. 5.2 finds the limit as the largest injection that forms no virtual cathode; here a
virtual cathode shows as emitted particles returning to the cathode (`return_fraction`,
current to the cathode plane over the emitted current).  Below the limit the whole
emission reaches the anode.  (Near the axis the anode current density then exceeds the
emitted one by several per cent: the electrodes short out the beam's radial electric
field but not its magnetic one, which pinches it; a guide field bz removes that.)"""
import math

import numpy as np

from . import pic
from workloads.bwo import EPS0, MU0, C0, QE, ME
from workloads.meshes import diode_mesh


def classical_limit(V, gap):
    """Non-relativistic planar Child-Langmuir current density (A/m^2)."""
    return 4.0 * EPS0 / 9.0 * math.sqrt(2.0 * abs(QE) / ME) * V ** 1.5 / gap ** 2


def run(V=1e5, gap=1e-2, radius=7e-2, r_emit=6e-2, n_tri=35_000, per_step=500, over=1.0,
        settle_steps=8000, measure_steps=6000, r_measure=1e-2, precision=pic.PIC_FP32,
        mesh_seed=1001, seed=77, graph=True, sort_interval=16, capacity=4_000_000,
        history_every=500, bz=0.0):
    """Run the diode and return the anode current density within r_measure, averaged
    over measure_steps after settle_steps, with the run's figures (and the same density
    averaged over every history_every steps of the whole run, to show it settle)."""
    import torch
    nodes, tris, be, bt = diode_mesh(n_tri=n_tri, seed=mesh_seed, gap=gap, radius=radius)
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
    pic.pic_sim_set_emitter(sim, 2e-3 * gap, 0.0, r_emit, per_step, 0.0, 0.0, seed, QE, ME,
                            weight)
    anode = np.flatnonzero(z == gap)
    anode = anode[np.argsort(nodes[anode, 1])]
    cathode = np.flatnonzero(z == 0.0)
    inside = anode[nodes[anode, 1] <= r_measure]
    rho_edge = 0.5 * (nodes[inside[-1], 1] + nodes[anode[len(inside)], 1])
    torch.cuda.synchronize()
    # node charges are per radian (the ring normalisation q w / (2 pi))
    area = math.pi * rho_edge ** 2
    history = []
    q_center = q_anode = q_win = q_back = 0.0
    total = settle_steps + measure_steps
    for k in range(total):
        pic.pic_step(sim, 1)
        _, _, Qa = pic.pic_charges_get(sim)
        qc = Qa[inside].sum()
        q_win += qc
        if k >= settle_steps:
            q_center += qc
            q_anode += Qa[anode].sum()
            q_back += Qa[cathode].sum()
        if (k + 1) % history_every == 0:
            history.append(abs(2.0 * math.pi * q_win) / (history_every * dt) / area)
            q_win = 0.0
    d = pic.pic_diagnostics(sim)
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
           "n_tris": len(tris), "J_center_history": history, "history_every": history_every}
    pic.pic_sim_destroy(sim)
    pic.pic_mesh_destroy(mesh)
    return out
