"""One EM-PIC cycle in the order of Sec. 3, FP64.  Test infrastructure.

State at the start of step n: E^n (edges), B^{n-1/2} (faces), particle positions r^n
(triangle + barycentric lambda), momenta u^{n-1/2}, node charges Q^n.
  0. emission (optional): new particles at r^n with u^{n-1/2}, their charge added to Q^n
  1. B^{n+1/2} = B^{n-1/2} - dt D_curl E^n                        (Eq. full_d_dfl)
  2. gather E^n (+ a static field) and (B^{n+1/2} + B^{n-1/2})/2 at r^n, push (Boris or
     Vay), walk, scatter J^{n+1/2} (Eq. current) and Q^{n+1} (Eq. charge) (Secs. 3.2-3.4)
  3. E^{n+1} = E^n + dt M (D_curl^T star_mu^-1 B^{n+1/2} - J^{n+1/2}) (Eq. full_d_dal)
The auxiliary dual flux D^{n+1} = D^n + dt (D_curl^T star_mu^-1 B^{n+1/2} - J^{n+1/2}) is
carried for the discrete Gauss law check: D_div D^n - Q^n is constant in n (Sec. 3.5.2).
"""
import math

import numpy as np

from .operators import Mesh, hodge_eps, hodge_mu_inv, spai, dt_stable, field_energy
from . import particles as P
from . import sources as S


class OracleSim:
    def __init__(self, nodes, tris, bedges, btags, eps0=1.0, mu0=1.0, c=None,
                 level=2, drop_tol=1e-4, M=None):
        self.mesh = Mesh(nodes, tris, bedges, btags)
        self.eps0, self.mu0 = eps0, mu0
        self.c = c if c is not None else 1.0 / math.sqrt(eps0 * mu0)
        self.star_eps = hodge_eps(self.mesh, eps0)
        self.mu_inv = hodge_mu_inv(self.mesh, mu0)
        self.M = spai(self.mesh, self.star_eps, level, drop_tol) if M is None else M
        self.dt_max, self.lam_max = dt_stable(self.mesh, self.M, self.mu_inv)
        self.pm = P.PushMesh(self.mesh)
        m = self.mesh
        self.E = np.zeros(m.N1)
        self.B = np.zeros(m.N2)            # B^{n-1/2}
        self.D = np.zeros(m.N1)
        self.Q = np.zeros(m.N0)
        self.Q_prev = np.zeros(m.N0)
        self.J = np.zeros(m.N1)
        self.Qabs = np.zeros(m.N0)
        self.tri = np.zeros(0, np.int32)
        self.lam = np.zeros((0, 3))
        self.u = np.zeros((0, 3))
        self.qm = 0.0
        self.q_src = 0.0
        self.q = self.mass = self.weight = 0.0
        self.dt = None
        self.bz = 0.0
        self.pusher = P.BORIS   # velocity update of Eq. DLE: P.BORIS or P.VAY
        self.counters = np.zeros(3, np.int64)
        self.n = 0
        self.E_static = None    # static (gun) field added at the gather, or None
        self.emitter = None     # dict of emitted() arguments and the species, or None
        self.Q_born = np.zeros(self.mesh.N0)   # charge of emitted particles, per node
        self.sigma_e = self.sigma_m = None      # absorbing layer conductivities, or None

    def create(self, dt, bz=0.0):
        if dt > self.dt_max:
            raise ValueError("dt above the stable limit")
        self.dt, self.bz = float(dt), float(bz)

    def set_fields(self, E, B_half_prev):
        E = np.array(E, float)
        E[self.mesh.edge_tag == 1] = 0.0
        self.E = E
        self.B = np.array(B_half_prev, float)
        self.D = self.star_eps @ self.E

    def inject(self, z, rho, ur, up, uz, q, mass, weight):
        """Locate the particles, append them, and add their charge to Q^n."""
        if self.q_src != 0.0 and (q / mass != self.qm or weight * q / (2 * math.pi) != self.q_src):
            raise ValueError("one species per simulation")
        self.q, self.mass, self.weight = q, mass, weight
        self.qm = q / mass
        # ring normalisation: the 2D equations are the 3D ones divided by 2 pi
        self.q_src = weight * q / (2.0 * math.pi)
        tri, lam = P.locate(self.mesh, z, rho)
        if np.any(tri < 0):
            raise ValueError("particle outside the mesh")
        u = np.stack([ur, up, uz], 1).astype(float)
        P.deposit_charge(self.pm, tri, np.ascontiguousarray(lam), self.q_src, self.Q)
        self.tri = np.ascontiguousarray(np.concatenate([self.tri, tri]).astype(np.int32))
        self.lam = np.ascontiguousarray(np.concatenate([self.lam, lam]))
        self.u = np.ascontiguousarray(np.concatenate([self.u, u]))

    def set_static_field(self, E_static):
        """A static field (edge values, e.g. from sources.static_potential) added to E^n
        at the gather only: it drives the particles but takes no part in the leapfrog."""
        self.E_static = None if E_static is None else np.array(E_static, float)

    def set_emitter(self, z0, rho0, rho1, per_step, u_normal, u_thermal, seed, q, mass,
                    weight):
        """Emit per_step particles at the start of every step (sources.emitted, ids
        continuing the particle count)."""
        self.emitter = dict(z0=z0, rho0=rho0, rho1=rho1, per_step=int(per_step),
                            u_normal=u_normal, u_thermal=u_thermal, seed=int(seed), q=q,
                            mass=mass, weight=weight)

    def emit(self):
        em = self.emitter
        pids = np.arange(len(self.tri), len(self.tri) + em["per_step"])
        z, r, ur, up, uz = S.emitted(em["z0"], em["rho0"], em["rho1"], em["u_normal"],
                                     em["u_thermal"], em["seed"], pids)
        q0 = self.Q.copy()
        self.inject(z, r, ur, up, uz, em["q"], em["mass"], em["weight"])
        self.Q_born += self.Q - q0

    def set_loss(self, sigma_e, sigma_m):
        """Absorbing layer: electric conductivity per edge, magnetic per face.  The
        conduction terms of the two curl equations are time-centred, so with
        s = sigma dt / (2 eps0) (resp. sigma_m dt / (2 mu0)) each update becomes
        x <- (1 - s)/(1 + s) x + (lossless increment) / (1 + s)."""
        if sigma_e is None and sigma_m is None:
            self.sigma_e = self.sigma_m = None
            return
        m = self.mesh
        self.sigma_e = np.zeros(m.N1) if sigma_e is None else np.array(sigma_e, float)
        self.sigma_m = np.zeros(m.N2) if sigma_m is None else np.array(sigma_m, float)

    def _loss_factors(self, s):
        return (1.0 - s) / (1.0 + s), 1.0 / (1.0 + s)

    def field_b_half(self):
        """Eq. full_d_dfl (with the magnetic conduction term in a lossy layer)."""
        inc = -self.dt * (self.mesh.Dcurl @ self.E)
        if self.sigma_m is None:
            return self.B + inc
        a, b = self._loss_factors(self.sigma_m * self.dt / (2.0 * self.mu0))
        return a * self.B + b * inc

    def push_particles(self, B_half):
        m = self.mesh
        Bavg = 0.5 * (B_half + self.B)
        self.J = np.zeros(m.N1)
        Qn = np.zeros(m.N0)
        self.Qabs = np.zeros(m.N0)
        Eg = self.E if self.E_static is None else self.E + self.E_static
        cnt = P.push(self.pm, Eg, Bavg, self.bz, self.dt, self.qm, self.c, self.q_src,
                     self.tri, self.lam, self.u, self.J, Qn, self.Qabs, pusher=self.pusher)
        self.counters += cnt
        return Qn

    def field_e(self, B_half):
        """Eq. full_d_dal with [star_eps]^-1 replaced by the SPAI matrix M."""
        m = self.mesh
        f = m.free
        r = m.Dcurl.T @ (self.mu_inv * B_half) - self.J
        self.D[f] += self.dt * r[f]
        inc = self.dt * (self.M @ r[f])
        if self.sigma_e is None:
            self.E[f] += inc
        else:
            a, b = self._loss_factors(self.sigma_e[f] * self.dt / (2.0 * self.eps0))
            self.E[f] = a * self.E[f] + b * inc

    def step(self, n=1):
        for _ in range(n):
            if self.emitter is not None:
                self.emit()
            B_half = self.field_b_half()
            Qn = self.push_particles(B_half)
            self.field_e(B_half)
            self.B = B_half
            self.Q_prev, self.Q = self.Q, Qn
            self.n += 1

    # ---- diagnostics (Sec. 3.5, Sec. 5.1.1) ----
    def dce_residual(self):
        """(Q^{n+1} - Q^n + Q_absorbed)/dt + D_div J^{n+1/2}, per node (Eq. DCE)."""
        return (self.Q - self.Q_prev + self.Qabs) / self.dt + self.mesh.Ddiv @ self.J

    def dgl_residual(self):
        """D_div D^n - Q^n at nodes not on a conducting wall (Eq. DGL_RSD_REL), with the
        charge of emitted particles (born without a current) taken out of Q^n."""
        m = self.mesh
        f = m.free
        res = m.Ddiv[:, f] @ self.D[f] - (self.Q - self.Q_born)
        res[m.node_on_pec] = 0.0
        if self.sigma_e is not None:
            # conduction moves charge in a lossy layer: its nodes are left out
            lossy = np.zeros(m.N0, bool)
            lossy[m.edge_nodes[self.sigma_e > 0].ravel()] = True
            lossy[m.tris[self.sigma_m > 0].ravel()] = True
            res[lossy] = 0.0
        return res

    def field_energy(self):
        return field_energy(self.mesh, self.star_eps, self.mu_inv, self.E, self.B)

    def kinetic_energy(self):
        """Total kinetic energy of the macro-particles (3D), (gamma - 1) m c^2 w."""
        live = self.tri >= 0
        u2 = np.sum(self.u[live] ** 2, 1)
        gam = np.sqrt(1.0 + u2 / self.c ** 2)
        return float(np.sum((gam - 1.0)) * self.mass * self.weight * self.c ** 2)

    def positions(self):
        """Physical (z, rho) of live particles from (triangle, lambda)."""
        live = self.tri >= 0
        p = self.mesh.nodes[self.mesh.tris[self.tri[live]]]
        zr = np.einsum("nk,nkd->nd", self.lam[live], p)
        return zr[:, 0], zr[:, 1]
