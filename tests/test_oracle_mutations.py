"""Planted mistakes: each case copies one oracle routine (Python or the plain C step),
changes one term the way a slip would (a flipped sign, a dropped factor, a swapped index
or operand), and runs the pin that is meant to catch it; the pin must fail.  This shows
that the pins constrain the oracle where it matters, rather than only re-running it.

Everything runs on the CPU.  Python routines are recompiled from their source text with
the one change; the C step is rebuilt from a changed copy of its source in a temporary
folder.  The oracle itself is never edited, and every change is undone after its case.
"""
import importlib
import inspect
import subprocess
import textwrap

import numpy as np
import pytest

import workloads as W
from oracle import OracleSim
from oracle import mlp as OM
from oracle import operators as OO
from oracle import particles as OP
from oracle import sim as OS
from oracle import sources as OSrc
from oracle import port as OPort

TP = importlib.import_module("test_oracle_particles")
TO = importlib.import_module("test_oracle_operators")
TU = importlib.import_module("test_oracle_pushers")
TS = importlib.import_module("test_oracle_sources")
TM = importlib.import_module("test_oracle_mlp")
TL = importlib.import_module("test_oracle_layer")
TF = importlib.import_module("test_oracle_fields")
TPo = importlib.import_module("test_oracle_port")


def _patch_py(monkeypatch, owner, name, old, new, importers=()):
    """Replace owner.name (a function, or a method of a class) by its source with the
    single occurrence of ``old`` replaced by ``new``; also rebind the name in modules that
    imported it directly."""
    fn = inspect.getattr_static(owner, name)
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == 1, (name, old)
    ns = {}
    exec(compile(src.replace(old, new), "<planted %s>" % name, "exec"), fn.__globals__, ns)
    monkeypatch.setattr(owner, name, ns[name])
    for mod in importers:
        monkeypatch.setattr(mod, name, ns[name])


def _patch_c(monkeypatch, tmp_path, old, new):
    """Point the oracle's loader at a copy of particles.c with one change, built the way
    the oracle builds its own."""
    with open(OP._SRC) as f:
        src = f.read()
    assert src.count(old) == 1, old
    path = tmp_path / "particles.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / "_liboracle_planted.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o",
                           str(lib), str(path), "-lm"])
    monkeypatch.setattr(OP, "_SRC", str(path))
    monkeypatch.setattr(OP, "_LIB", str(lib))
    monkeypatch.setattr(OP, "_lib", None)


@pytest.fixture(scope="module")
def cavity():
    """The particle pins' cavity (800 triangles, seed 11), built with the unchanged
    operators; used only by cases that change the particle step or the cycle."""
    return OracleSim(*W.cavity_mesh(n_tri=800, seed=11))


def _guide():
    return OracleSim(*W.meshes.rect_mesh(16.0, 1.0, 6000, 21))


# (case, change in particles.c: old -> new, the pin that must fail)
C_CASES = [
    ("current: tail and head swapped",
     "J[m->tri_edges[3 * t + k]] += w * (ls[a] * le[b] - ls[b] * le[a]);",
     "J[m->tri_edges[3 * t + k]] += w * (ls[b] * le[a] - ls[a] * le[b]);",
     lambda cav: TP.test_current_is_line_integral_of_whitney_form(cav)),
    ("gather: the rho gradient used for E_z",
     "ez += Ee * (lam[a] * g[2 * b + 0] - lam[b] * g[2 * a + 0]);",
     "ez += Ee * (lam[a] * g[2 * b + 1] - lam[b] * g[2 * a + 1]);",
     lambda cav: TP.test_uniform_E_kick(cav, 0)),
    ("gather: B_phi without the 1/A of the 2-form",
     "double Bf[3] = {0.0, Bavg[t] / area[t], bz};",
     "double Bf[3] = {0.0, Bavg[t], bz};",
     lambda cav: TP.test_rotational_field_fixes_faraday_sign_and_time_centred_B()),
    ("gather: E_rho with the wrong sign",
     "er += Ee * (lam[a] * g[2 * b + 1] - lam[b] * g[2 * a + 1]);",
     "er -= Ee * (lam[a] * g[2 * b + 1] - lam[b] * g[2 * a + 1]);",
     lambda cav: TP.test_uniform_E_kick(cav, 1)),
    ("gather: guide field B_z with the wrong sign",
     "double Bf[3] = {0.0, Bavg[t] / area[t], bz};",
     "double Bf[3] = {0.0, Bavg[t] / area[t], -bz};",
     lambda cav: TP.test_boris_gyration_closed_form()),
    ("walk: crossing parameter with the wrong sign",
     "double s = l[k] / (l[k] - le[k]);",
     "double s = l[k] / (le[k] - l[k]);",
     lambda cav: TP.test_walk_reaches_the_straight_line_endpoint(cav)),
    ("Boris: s = 2t without the 1/(1 + t^2)",
     "sv[i] = 2.0 * tv[i] / (1.0 + t2);",
     "sv[i] = 2.0 * tv[i];",
     lambda cav: TU.test_pure_magnetic_field_rotates_by_the_closed_form_angle(OP.BORIS)),
    ("Boris: gamma from u^{n-1/2} instead of u after the half kick",
     "double gam = sqrt(1.0 + dot3(um, um) / (c * c));",
     "double gam = sqrt(1.0 + dot3(u, u) / (c * c));",
     lambda cav: TU.test_boris_solves_the_momentum_mean_form(0.2)),
    ("cross product: one component with the wrong sign",
     "o[1] = a[2] * b[0] - a[0] * b[2];",
     "o[1] = a[0] * b[2] - a[2] * b[0];",
     lambda cav: TU.test_boris_solves_the_momentum_mean_form(0.01)),
    ("Vay: tau^2 enters sigma with the wrong sign",
     "double sigma = 1.0 + dot3(up, up) / (c * c) - tau2;",
     "double sigma = 1.0 + dot3(up, up) / (c * c) + tau2;",
     lambda cav: TU.test_vay_solves_the_velocity_mean_form(0.2)),
    ("pusher switch ignored inside the step",
     "if (pusher == 1) kick_vay(u, Ef, Bf, h, c, out);",
     "if (pusher == 2) kick_vay(u, Ef, Bf, h, c, out);",
     lambda cav: TU.test_cycle_uses_the_selected_pusher()),
    ("h = q dt / m: a whole step in each half kick",
     "const double h = 0.5 * qm * dt;",
     "const double h = qm * dt;",
     lambda cav: TP.test_uniform_E_kick(cav, 1)),
    ("rotate-back: the sine with the wrong sign",
     "double uphi = -sn * up[0] + cs * up[1];",
     "double uphi = sn * up[0] + cs * up[1];",
     lambda cav: TP.test_boris_gyration_closed_form()),
    ("move with u^{n-1/2} instead of u^{n+1/2}",
     "double vr = up[0] / gn, vp = up[1] / gn, vz = up[2] / gn;",
     "double vr = u[3 * p] / gn, vp = u[3 * p + 1] / gn, vz = u[3 * p + 2] / gn;",
     lambda cav: TP.test_boris_gyration_closed_form()),
    ("walk: the shared nodes' lambdas swapped in the neighbour",
     "if (nn[k] == gi) ln[k] = lc[i];",
     "if (nn[k] == gi) ln[k] = lc[j];",
     lambda cav: TP.test_walk_reaches_the_straight_line_endpoint(cav)),
    ("walk: the first crossing found, not the nearest",
     "if (s < sx) { sx = s; kx = k; }",
     "if (kx < 0) { sx = s; kx = k; }",
     lambda cav: TP.test_multi_cell_current_is_the_line_integral_over_the_crossed_cells(cav)),
    ("charge: the new position's nodes given the old lambdas",
     "for (int k = 0; k < 3; k++) ORACLE_ATOMIC Q[nn[k]] += q_src * l[k];",
     "for (int k = 0; k < 3; k++) ORACLE_ATOMIC Q[nn[k]] += q_src * lam[3 * p + k];",
     lambda cav: TP.test_dce_exact_with_multi_cell_crossings(cav)),
    ("charge at injection: each node given its neighbour's lambda",
     "Q[tri_nodes[3 * t + k]] += q_src * lam[3 * p + k];",
     "Q[tri_nodes[3 * t + k]] += q_src * lam[3 * p + (k + 1) % 3];",
     lambda cav: TP.test_dce_exact_with_multi_cell_crossings(cav)),
    ("walk: no cap on the crossings of one step",
     "if (nb < 0 || ncross + 1 >= max_cross) {",
     "if (nb < 0) {",
     lambda cav: TP.test_walk_cap_removes_the_particle_and_books_its_charge(cav)),
    ("walk: the rest of the displacement scaled by s, not 1 - s",
     "d[0] *= (1.0 - sx);",
     "d[0] *= sx;",
     lambda cav: TP.test_walk_reaches_the_straight_line_endpoint(cav)),
    ("edges: tail and head taken the other way round",
     "if (nodes3[i] < nodes3[j]) { *a = i; *b = j; }",
     "if (nodes3[i] > nodes3[j]) { *a = i; *b = j; }",
     lambda cav: TP.test_uniform_E_kick(cav, 0)),
    ("wall: the absorbed charge not booked",
     "for (int k = 0; k < 3; k++) ORACLE_ATOMIC Qabs[nn[k]] += q_src * lc[k];",
     "for (int k = 0; k < 3; k++) ORACLE_ATOMIC Qabs[nn[k]] += 0.0 * lc[k];",
     lambda cav: TP.test_absorbed_charge_enters_dce(cav)),
]


@pytest.mark.parametrize("case", C_CASES, ids=[c[0] for c in C_CASES])
def test_planted_mistake_in_the_particle_step_fails_its_pin(case, cavity, monkeypatch,
                                                              tmp_path):
    _, old, new, pin = case
    _patch_c(monkeypatch, tmp_path, old, new)
    with pytest.raises(AssertionError):
        pin(cavity)


def _recompute_m3(monkeypatch):
    monkeypatch.setattr(OO, "_M3", np.array([[[OO._moment3(i, j, k) for k in range(3)]
                                              for j in range(3)] for i in range(3)]))


# (case, owner, routine, old -> new, modules that imported the routine by name, the pin
#  that must fail, follow-up after the change or None)
PY_CASES = [
    ("moments: (a+b+c+1)! in the denominator", OO, "_moment3",
     "math.factorial(5)", "math.factorial(4)", (),
     lambda cav: TO.test_hodge_eps_by_quadrature(1), _recompute_m3),
    ("star_eps: one term's moment indices swapped", OO, "local_hodge_eps",
     "G[ar, b1, a2] * _M3[a1, b2, m]", "G[ar, b1, a2] * _M3[b1, a2, m]", (TO,),
     lambda cav: TO.test_hodge_eps_by_quadrature(2), None),
    ("star_eps: the rho weight left out", OO, "local_hodge_eps",
     "acc += rho[:, m] * (", "acc += (", (TO,),
     lambda cav: TO.test_hodge_eps_constant_rho_textbook(), None),
    ("star_mu^-1: the sum of the node rho instead of the mean", OO, "hodge_mu_inv",
     "[:, :, 1].mean(1)", "[:, :, 1].sum(1)", (TO, OS),
     lambda cav: TO.test_hodge_mu_by_quadrature(1), None),
    ("mesh: grad(lambda) with the wrong sign", OO.Mesh, "__init__",
     "g[:, k, 0] = (y[:, a] - y[:, b]) / (2 * self.area)",
     "g[:, k, 0] = (y[:, b] - y[:, a]) / (2 * self.area)", (),
     lambda cav: TO.test_gradients_and_area(1), None),
    ("mesh: D_curl oriented clockwise", OO.Mesh, "__init__",
     "self.dcurl_sign = np.where(i1 < i2, 1, -1)",
     "self.dcurl_sign = np.where(i1 > i2, 1, -1)", (),
     lambda cav: TP.test_rotational_field_fixes_faraday_sign_and_time_centred_B(), None),
    ("mesh: D_div positive at the head", OO.Mesh, "__init__",
     "(np.concatenate([np.ones(self.N1), -np.ones(self.N1)]),",
     "(np.concatenate([-np.ones(self.N1), np.ones(self.N1)]),", (),
     lambda cav: TS.test_charge_conservation_with_particles_born_every_step(), None),
    ("SPAI: not symmetrised", OO, "spai",
     "return (0.5 * (M + M.T)).tocsr()", "return M.tocsr()", (TO, OS),
     lambda cav: TO.test_spai_quality_and_symmetry(), None),
    ("SPAI: each column fitted to its pattern's first unit vector", OO, "spai",
     "rhs = (R == j).astype(float)", "rhs = (R == S[0]).astype(float)", (TO, OS),
     lambda cav: TO.test_spai_quality_and_symmetry(), None),
    ("stable step 1/sqrt(lambda_max)", OO, "dt_stable",
     "return 2.0 / math.sqrt(lam), lam", "return 1.0 / math.sqrt(lam), lam", (TO, OS),
     lambda cav: TO.test_dt_stable_matches_eigensolver(), None),
    ("location: lambda over the area instead of twice the area", OP, "barycentric",
     "/ (2.0 * mesh.area[t])", "/ mesh.area[t]", (TO,),
     lambda cav: TP.test_locate_by_brute_force(), None),
    ("location: one product of the signed area with swapped nodes", OP, "barycentric",
     "lam[:, k] = ((p[:, a, 0] - z) * (p[:, b, 1] - rho)",
     "lam[:, k] = ((p[:, b, 0] - z) * (p[:, a, 1] - rho)", (TO,),
     lambda cav: TP.test_locate_by_brute_force(), None),
    ("SPAI: one hop more than the pattern level", OO, "spai_pattern",
     "for _ in range(level):", "for _ in range(level + 1):", (),
     lambda cav: TO.test_spai_level0_closed_form(), None),
    ("stable step: curl-curl operator without star_mu^-1", OO, "curl_curl",
     "return (Dc.T @ sp.diags(mu_inv) @ Dc).tocsr()", "return (Dc.T @ Dc).tocsr()", (TO,),
     lambda cav: TF.test_stability_limit(OracleSim(*W.cavity_mesh())), None),
    ("field energy: magnetic part without the 1/2", OO, "field_energy",
     "0.5 * np.sum(mu_inv * B * B)", "np.sum(mu_inv * B * B)", (OS,),
     lambda cav: TF.test_field_energy_of_uniform_fields_closed_form(), None),
    ("field energy: electric part without star_eps", OO, "field_energy",
     "0.5 * E @ (star_eps @ E)", "0.5 * E @ E", (OS,),
     lambda cav: TF.test_field_energy_of_uniform_fields_closed_form(), None),
    ("kinetic energy: gamma m c^2 instead of (gamma - 1) m c^2", OS.OracleSim,
     "kinetic_energy", "np.sum((gam - 1.0))", "np.sum(gam)", (),
     lambda cav: TP.test_kinetic_energy_limits(cav), None),
    ("kinetic energy: the macro-particle weight left out", OS.OracleSim, "kinetic_energy",
     "* self.mass * self.weight * self.c ** 2", "* self.mass * self.c ** 2", (),
     lambda cav: TP.test_kinetic_energy_limits(cav), None),
    ("mesh: each triangle its own neighbour across an interior edge", OO.Mesh, "__init__",
     "self.nbr[et[both, 0], el[both, 0]] = et[both, 1]",
     "self.nbr[et[both, 0], el[both, 0]] = et[both, 0]", (),
     lambda cav: TP.test_walk_reaches_the_straight_line_endpoint(
         OracleSim(*W.cavity_mesh(n_tri=800, seed=11))), None),
    ("star_eps: local blocks assembled with rows for columns", OO, "hodge_eps",
     "c = np.tile(mesh.tri_edges, (1, 3)).ravel()",
     "c = np.repeat(mesh.tri_edges, 3, axis=1).ravel()", (TO, OS),
     lambda cav: TO.test_hodge_spd(), None),
    ("fields: tangential E kept on conductor edges", OS.OracleSim, "set_fields",
     "E[self.mesh.edge_tag == 1] = 0.0", "pass", (),
     lambda cav: TF.test_conducting_walls_short_the_tangential_field(), None),
    ("Gauss law: conductor nodes not left out", OS.OracleSim, "dgl_residual",
     "res[m.node_on_pec] = 0.0", "pass", (),
     lambda cav: TP.test_dgl_residual_constant(cav), None),
    ("layer: E increment without the 1/(1 + s)", OS.OracleSim, "field_e",
     "self.E[f] = a * self.E[f] + b * inc", "self.E[f] = a * self.E[f] + inc", (),
     lambda cav: TL.test_matched_uniform_conductor_scales_the_lossless_run(), None),
    ("layer: B increment without the 1/(1 + s)", OS.OracleSim, "field_b_half",
     "return a * self.B + b * inc", "return a * self.B + inc", (),
     lambda cav: TL.test_matched_uniform_conductor_scales_the_lossless_run(), None),
    ("emission: ids restart every step", OS.OracleSim, "emit",
     'pids = np.arange(len(self.tri), len(self.tri) + em["per_step"])',
     'pids = np.arange(em["per_step"])', (),
     lambda cav: TS.test_successive_emissions_continue_the_particle_ids(), None),
    ("draws: the half step dropped (0 becomes a possible draw)", OSrc, "uniforms",
     ".astype(np.float64) + 0.5) * 2.0 ** -53", ".astype(np.float64)) * 2.0 ** -53", (),
     lambda cav: TS.test_uniform_draws_stay_inside_the_open_interval_at_the_extremes(), None),
    ("emission: cosine for both transverse momenta", OSrc, "emitted",
     "up = u_thermal * r1 * np.sin(2.0 * math.pi * u[:, 2])",
     "up = u_thermal * r1 * np.cos(2.0 * math.pi * u[:, 2])", (),
     lambda cav: TS.test_emitted_transverse_momenta_are_independent_normals(), None),
    ("static field: node charge with the wrong sign", OSrc, "static_potential",
     "rhs = rhs + np.asarray(charge, float)[free]", "rhs = rhs - np.asarray(charge, float)[free]", (),
     lambda cav: TS.test_gauss_law_of_a_charged_shell_fixes_the_ring_normalisation(), None),
    ("cycle: B^{n+1/2} at the gather instead of the time-centred B", OS.OracleSim,
     "push_particles", "Bavg = 0.5 * (B_half + self.B)", "Bavg = B_half", (),
     lambda cav: TP.test_rotational_field_fixes_faraday_sign_and_time_centred_B(), None),
    ("cycle: Faraday's law with the wrong sign", OS.OracleSim, "field_b_half",
     "inc = -self.dt * (self.mesh.Dcurl @ self.E)",
     "inc = self.dt * (self.mesh.Dcurl @ self.E)", (),
     lambda cav: TP.test_rotational_field_fixes_faraday_sign_and_time_centred_B(), None),
    ("cycle: J enters Ampere's law with the wrong sign", OS.OracleSim, "field_e",
     "r = m.Dcurl.T @ (self.mu_inv * B_half) - self.J",
     "r = m.Dcurl.T @ (self.mu_inv * B_half) + self.J", (),
     lambda cav: TP.test_energy_balance_fixes_ring_normalisation(), None),
    ("cycle: the dual flux D not advanced", OS.OracleSim, "field_e",
     "self.D[f] += self.dt * r[f]", "self.D[f] += 0.0 * r[f]", (),
     lambda cav: TP.test_dgl_residual_constant(cav), None),
    ("cycle: ring charge without the 1/(2 pi)", OS.OracleSim, "inject",
     "self.q_src = weight * q / (2.0 * math.pi)", "self.q_src = weight * q", (),
     lambda cav: TP.test_energy_balance_fixes_ring_normalisation(), None),
    ("cycle: static field left out of the gather", OS.OracleSim, "push_particles",
     "Eg = self.E if self.E_static is None else self.E + self.E_static", "Eg = self.E", (),
     lambda cav: TS.test_static_field_drives_particles_but_not_the_leapfrog(), None),
    ("cycle: static field added to the leapfrog's E", OS.OracleSim, "set_static_field",
     "self.E_static = None if E_static is None else np.array(E_static, float)",
     "self.E_static = None; self.E = self.E + np.array(E_static, float)", (),
     lambda cav: TS.test_static_field_drives_particles_but_not_the_leapfrog(), None),
    ("emission: born charge not recorded", OS.OracleSim, "emit",
     "self.Q_born += self.Q - q0", "self.Q_born += 0.0 * (self.Q - q0)", (),
     lambda cav: TS.test_charge_conservation_with_particles_born_every_step(), None),
    ("layer: decay and increment factors swapped", OS.OracleSim, "_loss_factors",
     "return (1.0 - s) / (1.0 + s), 1.0 / (1.0 + s)",
     "return 1.0 / (1.0 + s), (1.0 - s) / (1.0 + s)", (),
     lambda cav: TL.test_uniform_conductivity_decays_a_curl_free_field_exactly(_guide()), None),
    ("splitmix64: shift 31 for 30", OSrc, "splitmix64",
     "z = (z ^ (z >> np.uint64(30))) * _M1", "z = (z ^ (z >> np.uint64(31))) * _M1", (),
     lambda cav: TS.test_splitmix64_published_outputs(), None),
    ("emission: uniform in rho instead of in area", OSrc, "emitted",
     "rho = np.sqrt(rho0 * rho0 + u[:, 0] * (rho1 * rho1 - rho0 * rho0))",
     "rho = rho0 + u[:, 0] * (rho1 - rho0)", (),
     lambda cav: TS.test_emitted_distributions(), None),
    ("static field: E = +grad phi", OSrc, "static_potential",
     "return phi, mesh.Ddiv.T @ phi", "return phi, -(mesh.Ddiv.T @ phi)", (),
     lambda cav: TS.test_static_potential_of_a_planar_gap_is_exact(), None),
    ("Child-Langmuir: exponent -1/2 for -1/4", OSrc, "child_langmuir_planar",
     "(x * (2.0 + x)) ** -0.25", "(x * (2.0 + x)) ** -0.5", (),
     lambda cav: TS.test_child_langmuir_limits(), None),
    ("network: GELU derivative without the tanh' term", OM, "gelu_grad",
     "return 0.5 * (1.0 + t) + 0.5 * z * dt", "return 0.5 * (1.0 + t)", (),
     lambda cav: TM.test_backward_matches_finite_differences(), None),
    ("network: bias gradient averaged over the batch", OM, "backward",
     "dbs[l] = g.sum(0)", "dbs[l] = g.mean(0)", (),
     lambda cav: TM.test_backward_matches_finite_differences(), None),
    ("network: activation after the output layer", OM, "forward",
     "a = gelu(z) if l < L - 1 else z", "a = gelu(z)", (),
     lambda cav: TM.test_single_layer_is_the_affine_map(), None),
    ("Adam: no bias correction of the second moment", OM, "adam",
     "vh = vv / (1 - b2 ** step)", "vh = vv", (),
     lambda cav: TM.test_adam_first_step_is_signed_learning_rate(), None),
    ("Adam: first moment without the (1 - b1) weight", OM, "adam",
     "mm += (1 - b1) * g", "mm += g", (),
     lambda cav: TM.test_adam_first_step_is_signed_learning_rate(), None),
    ("network: loss summed instead of averaged", OM, "loss",
     "return np.mean((y - t) ** 2)", "return np.sum((y - t) ** 2)", (),
     lambda cav: TM.test_backward_matches_finite_differences(), None),
    ("Adam: no bias correction of the first moment", OM, "adam",
     "mh = mm / (1 - b1 ** step)", "mh = mm", (),
     lambda cav: TM.test_adam_first_step_is_signed_learning_rate(), None),
    ("port: the rho of the flux element left out", OPort, "port_power",
     "* r for r in (a, 0.5 * (a + b), b)]", "for r in (a, 0.5 * (a + b), b)]", (),
     lambda cav: TPo.test_uniform_fields_give_the_closed_form(_port_guide(), 0.1, 0.37), None),
    ("port: the W1 terms of an edge in the wrong order", OPort, "e_rho",
     "(lam[a] * g[b, 1] - lam[b] * g[a, 1])", "(lam[b] * g[a, 1] - lam[a] * g[b, 1])", (),
     lambda cav: TPo.test_uniform_fields_give_the_closed_form(_port_guide(), 0.0, 0.5), None),
    ("port: B_phi without 1/A", OPort, "port_power",
     "bphi = B[t] / mesh.area[t]", "bphi = B[t]", (),
     lambda cav: TPo.test_uniform_fields_give_the_closed_form(_port_guide(), 0.0, 0.5), None),
    ("port: the chord's midpoint weighted 2 instead of 4", OPort, "port_power",
     "(f[0] + 4.0 * f[1] + f[2])", "(f[0] + 2.0 * f[1] + f[2])", (),
     lambda cav: TPo.test_linear_in_z_field_gives_its_value_at_the_plane(_port_guide()), None),
]


def _port_guide():
    return OO.Mesh(*W.rect_mesh(1.0, 0.5, 1200, 17))


@pytest.mark.parametrize("case", PY_CASES, ids=[c[0] for c in PY_CASES])
def test_planted_mistake_in_a_python_routine_fails_its_pin(case, cavity, monkeypatch):
    _, owner, name, old, new, importers, pin, follow = case
    _patch_py(monkeypatch, owner, name, old, new, importers)
    if follow is not None:
        follow(monkeypatch)
    with pytest.raises(AssertionError):
        pin(cavity)
