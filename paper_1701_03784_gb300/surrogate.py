"""Surrogate of the ripple sweep: outputs of batched simulations, and an ensemble of
networks (pic_mlp_*) trained on them that answers only where its members agree.

Outputs of one simulated instance (``batch_outputs``), from the azimuthal magnetic field
sampled on the device every ``every`` steps (pic_sim_set_probes):
  * envelope: log10 of the magnetic energy (sum over faces of B_f^2 / 2 times the diagonal
    star_mu^-1 coefficient rho_bar / (mu0 A)) past ``out_z`` in the instance's own frame,
    averaged over 32 equal windows of the run;
  * frequency: the peak of the spectrum of B at a probe face.
The network input is the instance's parameters (ripple depth, period, number of periods,
beam voltage, beam current, guide field), scaled to [-1, 1] over the sweep's ranges.
"""
import math

import numpy as np

from . import pic
from .batch import union

N_ENV = 32
# feature ranges: depth (m), period (m), periods, voltage (V), current (A), guide field (T)
FEATURE_LO = np.array([0.2e-2, 1.4e-2, 8.0, 300e3, 0.0, 1.5])
FEATURE_HI = np.array([0.6e-2, 2.0e-2, 16.0, 500e3, 6e3, 3.5])
SIZES = (6, 256, 256, 256, 256, N_ENV + 1)


def features(params):
    """Rows of (depth, period, n_periods, voltage, current, bz) scaled to [-1, 1]."""
    p = np.atleast_2d(np.asarray(params, float))
    return 2.0 * (p - FEATURE_LO) / (FEATURE_HI - FEATURE_LO) - 1.0


def _face_geometry(nodes, tris):
    p = nodes[tris]
    area = 0.5 * np.abs((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                        - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    return p.mean(1), p[:, :, 1].mean(1), area


def batch_outputs(instances, dt, bz, steps, every, q, m, w, eps0, mu0, c, sort_interval=16):
    """Simulate the instances together (one simulation of their mesh union) for ``steps``
    steps from zero fields and return (envelopes n x 32, frequencies n, in Hz).

    Each instance needs, besides its mesh and particles, ``out_z`` (where the measured
    region starts) and ``probe`` (a (z, rho) point), both in its own frame."""
    assert steps % (every * N_ENV) == 0
    u = union(instances)
    mesh = pic.pic_mesh_create(u["nodes"], u["tris"], u["be"], u["bt"], eps0=eps0, mu0=mu0, c=c,
                               precision=pic.PIC_FP32)
    dt_max = pic.pic_spai_build(mesh, 2, 1e-4)
    if dt > dt_max:
        raise ValueError("time step %.3g above the union's stable step %.3g" % (dt, dt_max))
    info = pic.pic_mesh_info(mesh)
    sim = pic.pic_sim_create(mesh, dt, bz, len(u["z"]) + 1024)
    pic.pic_sim_set_sort_interval(sim, sort_interval)
    pic.pic_sim_set_graph(sim, True)
    pic.pic_fields_set(sim, np.zeros(info["n_edges"]), np.zeros(info["n_tris"]))
    pic.pic_particles_inject(sim, u["z"], u["r"], u["ur"], u["up"], u["uz"], q, m, w)

    cen, rho_bar, area = _face_geometry(u["nodes"], u["tris"])
    coef = 0.5 * rho_bar / (mu0 * area)
    n = len(instances)
    inst = np.repeat(np.arange(n), np.diff(u["tri_off"]))
    z_local = cen[:, 0] - u["shift"][inst]
    out = z_local >= np.array([x["out_z"] for x in instances])[inst]
    probe = np.empty(n, np.int64)
    for i, x in enumerate(instances):
        t0, t1 = u["tri_off"][i], u["tri_off"][i + 1]
        d = (z_local[t0:t1] - x["probe"][0]) ** 2 + (cen[t0:t1, 1] - x["probe"][1]) ** 2
        probe[i] = t0 + int(np.argmin(d))
    samples = steps // every
    # recorded on the device every `every` steps: group i the magnetic energy past out_z
    # of instance i, group n + i the probe face's B
    faces = np.flatnonzero(out)
    pic.pic_sim_set_probes(sim, np.concatenate([faces, probe]),
                           np.concatenate([inst[faces], n + np.arange(n)]),
                           np.concatenate([coef[faces], np.ones(n)]),
                           np.array([2] * n + [1] * n), capacity=samples, every=every)
    pic.pic_step(sim, steps)
    rec, dropped = pic.pic_probes_read(sim)
    assert len(rec) == samples and dropped == 0
    energy = rec[:, :n].T
    bprobe = rec[:, n:].T
    env = np.log10(energy.reshape(n, N_ENV, samples // N_ENV).mean(2) + 1e-300)
    spec = np.abs(np.fft.rfft(bprobe - bprobe.mean(1, keepdims=True), axis=1))
    k = 1 + np.argmax(spec[:, 1:], axis=1)
    freq = k / (samples * every * dt)
    pic.pic_sim_destroy(sim)
    return env, freq


class Ensemble:
    """n_members networks trained on the same data from different starting points and
    minibatch draws.  Targets are standardised per output; predictions are the members'
    mean, and the spread of the output power (mean of 10^envelope) across members
    decides whether the ensemble answers."""

    def __init__(self, members=5, sizes=SIZES, max_batch=256, seed=0):
        self.members = members
        self.sizes = sizes
        self.seed = seed
        self.net = pic.pic_mlp_create(members, sizes, max_batch)
        rng = np.random.default_rng(seed)
        params = []
        for _ in range(members):
            p = []
            for k, n in zip(sizes[:-1], sizes[1:]):
                lim = 1.0 / math.sqrt(k)
                p.append(rng.uniform(-lim, lim, n * k))
                p.append(np.zeros(n))
            params.append(np.concatenate(p))
        pic.pic_mlp_params_set(self.net, np.stack(params))
        self.mu = self.sd = None

    def fit(self, X, Y, steps, batch=128, lr=1e-3, seed=1):
        import torch
        self.mu = Y.mean(0)
        self.sd = Y.std(0) + 1e-12
        Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
        Td = torch.tensor((Y - self.mu) / self.sd, dtype=torch.float32, device="cuda")
        return pic.pic_mlp_train(self.net, Xd, Td, batch, steps, lr=lr, seed=seed)

    def predict(self, X, tensor_cores=True):
        """(mean prediction, per-member predictions) in the targets' units."""
        import torch
        Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
        Y = pic.pic_mlp_forward(self.net, Xd, tensor_cores=tensor_cores).cpu().numpy()
        Y = Y * self.sd + self.mu
        return Y.mean(0), Y

    @staticmethod
    def power(Y):
        """Output power of predictions (last axis: 32 envelope samples, frequency)."""
        return (10.0 ** Y[..., :N_ENV]).mean(-1)

    def answer(self, X, tol=0.05, tensor_cores=True):
        """(mean prediction, mask of the rows whose members' output powers agree within
        tol relative spread: std / mean)."""
        mean, Ym = self.predict(X, tensor_cores)
        P = self.power(Ym)
        spread = P.std(0) / np.abs(P.mean(0))
        return mean, spread <= tol, spread
