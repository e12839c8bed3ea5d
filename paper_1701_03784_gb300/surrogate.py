"""Surrogate of the ripple sweep: outputs of batched simulations, and an ensemble of
networks (pic_mlp_*) trained on them that answers only where its members agree.

Outputs of one simulated instance (``batch_outputs``), from the output-port power recorded
on the device every ``every`` steps (pic_sim_set_ports: the Poynting flux through the
instance's output plane, a few mm inside its output end):
  * envelope: the port power (MW) averaged over 32 equal windows of the run;
  * frequency: the strongest oscillation of the port power between 4 and 100 GHz after
    the arrival (what the structure rings at once the beam has reached the end;
    ``ringing_frequency``).
Each run starts from zero fields with the instance's beam filling its slow-wave section,
so the record is one pulse: the power rises while the beam approaches the output plane
and, once the beam reaches the absorbing end, rings with reflections whose net flux runs
both ways.  The power the surrogate answers for is the mean over the arrival, the first
N_ARRIVAL windows (the rising part of every instance's pulse; its run-to-run scatter over
mesh realisations is about 0.3%, where that of the whole run's mean, net of the ringing,
is twice as large and follows the beam parameters far less smoothly).
The networks learn the outputs as ``targets`` lays them out: the log of the arrival
power over the square of the beam current, the other windows relative to the arrival
power, and the frequency.
The network input is the instance's parameters (ripple depth, period, number of periods,
beam voltage, beam current, guide field), scaled to [-1, 1] over the sweep's ranges.
"""
import math

import numpy as np

from . import pic
from .batch import union

N_ENV = 32
N_ARRIVAL = 12
I_REF = 1e3      # A
N_OUT = N_ENV + 1
# feature ranges: depth (m), period (m), periods, voltage (V), current (A), guide field (T)
FEATURE_LO = np.array([0.2e-2, 1.4e-2, 8.0, 300e3, 0.0, 1.5])
FEATURE_HI = np.array([0.6e-2, 2.0e-2, 16.0, 500e3, 6e3, 3.5])
SIZES = (6, 256, 256, 256, 256, N_OUT)


def targets(env, freq, current):
    """Network outputs of simulated runs: log10 of the arrival power (the mean of the
    first N_ARRIVAL windows, MW) over (current / I_REF)^2 (the beam's own field carries a
    power that goes with the square of its current: what is left varies over a range six
    times narrower), windows 1..31 over the arrival power (window 0 follows from the
    arrival's sum), and the frequency in GHz."""
    env = np.atleast_2d(env)
    arrival = env[:, :N_ARRIVAL].mean(1)
    if np.any(arrival <= 0):
        raise ValueError("a run whose arrival power is not positive")
    scale = (np.asarray(current, float) / I_REF) ** 2
    return np.ascontiguousarray(np.column_stack([np.log10(arrival / scale),
                                                 env[:, 1:] / arrival[:, None],
                                                 np.asarray(freq) * 1e-9]))


def arrival_power(Y, current):
    """Arrival power (MW) of outputs Y laid out as ``targets`` for beams of that current."""
    return 10.0 ** np.asarray(Y)[..., 0] * (np.asarray(current, float) / I_REF) ** 2


def envelope(Y, current):
    """The 32-window power envelope (MW) of outputs Y (the inverse of ``targets``)."""
    Y = np.asarray(Y)
    arrival = arrival_power(Y, current)[..., None]
    rest = Y[..., 1:N_ENV]
    first = N_ARRIVAL - rest[..., :N_ARRIVAL - 1].sum(-1, keepdims=True)
    return arrival * np.concatenate([first, rest], -1)


def features(params):
    """Rows of (depth, period, n_periods, voltage, current, bz) scaled to [-1, 1]."""
    p = np.atleast_2d(np.asarray(params, float))
    return 2.0 * (p - FEATURE_LO) / (FEATURE_HI - FEATURE_LO) - 1.0


def _face_geometry(nodes, tris):
    p = nodes[tris]
    area = 0.5 * np.abs((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1])
                        - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1]))
    return p.mean(1), p[:, :, 1].mean(1), area


def ringing_frequency(P, dt, f_max=100e9, f_min=4e9, pad=8):
    """Frequency (Hz) of the strongest oscillation in (f_min, f_max] of each row of P (power
    samples dt apart): the peak of the magnitude spectrum of the row less its least-squares
    line, under a Hann window and zero-padded to pad times the next power of two, refined
    by the parabola through the log magnitudes of the peak bin and its two neighbours."""
    P = np.atleast_2d(np.asarray(P, float))
    m = P.shape[1]
    nfft = pad * (1 << int(math.ceil(math.log2(m))))
    s = np.linspace(-1.0, 1.0, m)
    slope = (P * s).sum(1, keepdims=True) / (s * s).sum()
    x = (P - P.mean(1, keepdims=True) - slope * s) * np.hanning(m)
    mag = np.abs(np.fft.rfft(x, nfft, axis=1))
    f = np.fft.rfftfreq(nfft, dt)
    band = (f > f_min) & (f <= f_max)
    lo = int(np.flatnonzero(band)[0])
    hi = int(np.flatnonzero(band)[-1])
    k = lo + np.argmax(mag[:, lo:hi + 1], axis=1)
    k = np.clip(k, lo + 1, hi - 1)
    rows = np.arange(len(P))
    a, b, c = (np.log(mag[rows, k + d] + 1e-300) for d in (-1, 0, 1))
    den = a - 2.0 * b + c
    delta = np.where(den < 0, 0.5 * (a - c) / np.where(den < 0, den, -1.0), 0.0)
    return (k + np.clip(delta, -0.5, 0.5)) * (f[1] - f[0])


def batch_outputs(instances, dt, bz, steps, every, q, m, w, eps0, mu0, c, sort_interval=16,
                  port_offset=4.93e-3, f_max=100e9):
    """Simulate the instances together (one simulation of their mesh union) for ``steps``
    steps from zero fields and return (envelopes n x 32 in MW, frequencies n in Hz, the
    port power records n x steps/every in W).

    Each instance needs, besides its mesh and particles, ``z_end`` (its output end) and
    ``r_out`` (the output guide's radius), in its own frame; its port plane is
    port_offset inside the output end.  The plane keeps several cells from the absorbing
    end: in the first row of cells next to it, the fields carry the near field of the
    charge that absorbed particles leave on that boundary, and the flux there changes by up
    to 13% from one jittered mesh to another (a few mm in, by about 1%)."""
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
    n = len(instances)
    samples = steps // every
    zp = np.array([u["shift"][i] + x["z_end"] - port_offset for i, x in enumerate(instances)])
    r_out = np.array([x["r_out"] for x in instances]) * (1.0 - 1e-9)
    pic.pic_sim_set_ports(sim, zp, 0.0, r_out, capacity=samples, every=every)
    pic.pic_step(sim, steps)
    rec, dropped = pic.pic_ports_read(sim)
    assert len(rec) == samples and dropped == 0
    P = rec.T
    env = P.reshape(n, N_ENV, samples // N_ENV).mean(2) / 1e6
    freq = ringing_frequency(P[:, samples * N_ARRIVAL // N_ENV:], every * dt, f_max)
    pic.pic_sim_destroy(sim)
    return env, freq, P


class Ensemble:
    """n_members networks trained on the same data from different starting points and
    minibatch draws.  Targets are standardised per output, the arrival power's scaled up
    by ``power_gain`` (its weight in the squared loss is power_gain^2: one output among
    33, and the one the ensemble answers for); predictions are the members' mean, and the
    spread of the arrival power across members decides whether the ensemble answers."""

    def __init__(self, members=5, sizes=SIZES, max_batch=256, seed=0, power_gain=16.0):
        self.members = members
        self.power_gain = power_gain
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

    def fit(self, X, Y, steps, batch=128, lr=1e-3, seed=1, chunks=8):
        """Adam on the device (pic_mlp_train) for ``steps`` minibatches in ``chunks`` calls,
        the learning rate of chunk k lr (1 + cos(pi (k + 1/2) / chunks)) / 2 (a cosine
        decay; the optimiser's moments and step count carry over between calls).  Returns
        each member's loss on its last minibatch."""
        import torch
        self.mu = Y.mean(0)
        self.sd = Y.std(0) + 1e-12 * (np.abs(Y).max() + 1.0)
        self.sd[0] /= self.power_gain
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        Td = torch.from_numpy(np.ascontiguousarray((Y - self.mu) / self.sd,
                                                   dtype=np.float32)).cuda()
        bounds = np.linspace(0, steps, chunks + 1).astype(int)
        loss = None
        for k in range(chunks):
            n = int(bounds[k + 1] - bounds[k])
            if n:
                rate = lr * 0.5 * (1.0 + math.cos(math.pi * (k + 0.5) / chunks))
                loss = pic.pic_mlp_train(self.net, Xd, Td, batch, n, lr=rate, seed=seed)
        return loss

    def predict(self, X, tensor_cores=True):
        """(mean prediction, per-member predictions) in the targets' units."""
        import torch
        Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).cuda()
        Y = pic.pic_mlp_forward(self.net, Xd, tensor_cores=tensor_cores).cpu().numpy()
        Y = Y * self.sd + self.mu
        return Y.mean(0), Y

    @staticmethod
    def power(Y):
        """Arrival power over (current / I_REF)^2 of outputs laid out as ``targets`` (the
        current is an input, so relative spreads and errors are those of the power)."""
        return 10.0 ** np.asarray(Y)[..., 0]

    def answer(self, X, tol=0.05, tensor_cores=True):
        """(mean prediction, mask of the rows whose members' arrival powers agree within
        tol relative spread: std / |mean|, the spread)."""
        mean, Ym = self.predict(X, tensor_cores)
        P = self.power(Ym)
        spread = P.std(0) / np.abs(P.mean(0))
        return mean, spread <= tol, spread

    @staticmethod
    def calibrate(spread, err, target=0.05, margin=0.8):
        """The largest spread threshold under which every calibration row's error stays
        below margin * target (the gate then answers only where the members agree that
        well); 0 if none does."""
        order = np.argsort(spread)
        ok = np.cumsum(err[order] > margin * target) == 0
        return float(spread[order][ok].max()) if ok.any() else 0.0


def simulate(make_instance, ids, bz, steps, every, dt, q, m, w, eps0, mu0, c, scale=1.0,
             pool=None):
    """PIC outputs of the instances ``make_instance(i)`` for i in ids, simulated as one
    union under the guide field bz: (input rows n x 6 in physical units, targets n x N_OUT,
    port power records n x steps/every in W, seconds spent simulating).  The current input
    is the instance's effective current over ``scale``, the current of the full-size beam
    the instance's reduced beam stands for (same velocity, scale of the charge)."""
    import time
    ins = pool.map(make_instance, ids) if pool is not None else [make_instance(i) for i in ids]
    t0 = time.time()
    env, freq, P = batch_outputs(ins, dt, bz, steps, every, q, m, w, eps0, mu0, c)
    seconds = time.time() - t0
    rows = np.array([[x["params"]["depth"], x["params"]["period"], x["params"]["n_periods"],
                      x["params"]["voltage"], x["current_eff"] / scale, bz] for x in ins])
    return rows, targets(env, freq, rows[:, 4]), P, seconds


def study(make_instance, n_train, n_val, n_test, steps, every, dt, q, m, w, eps0, mu0, c,
          scale=1.0, per_union=64, train_steps=8000, power_gain=16.0, members=5, pool=None,
          bz_range=(1.5, 3.5), target=0.05, margin=0.8, seed=7):
    """Surrogate from simulated runs: instances 0 .. n_train + n_val + n_test - 1 in unions of
    per_union, the training unions' guide fields on an even grid over bz_range and the
    validation and held-out unions' drawn inside it; the ensemble trained on the training
    runs, its answer gate calibrated on the validation runs (``Ensemble.calibrate``), and
    its errors on the held-out runs.  Returns a dict: rows, Y, records, the ensemble, the
    gate's threshold and, for the held-out runs, the arrival-power and frequency errors,
    the spreads and the answered mask, with the seconds spent simulating and training."""
    import time
    import torch
    total = n_train + n_val + n_test
    n_tb = -(-n_train // per_union)
    rows, Y, rec, sim_s = [], [], [], 0.0
    for b0 in range(0, total, per_union):
        if b0 < n_train:
            bz = bz_range[0] + (bz_range[1] - bz_range[0]) * (b0 // per_union) / max(n_tb - 1, 1)
        else:
            bz = float(np.random.default_rng(100000 + b0).uniform(*bz_range))
        r, y, P, s = simulate(make_instance, list(range(b0, min(b0 + per_union, total))), bz,
                              steps, every, dt, q, m, w, eps0, mu0, c, scale, pool)
        rows.append(r)
        Y.append(y)
        rec.append(P.astype(np.float32))
        sim_s += s
    rows, Y, rec = np.concatenate(rows), np.concatenate(Y), np.concatenate(rec)
    X = features(rows)
    tr, va, te = (slice(0, n_train), slice(n_train, n_train + n_val),
                  slice(n_train + n_val, total))
    ens = Ensemble(members, SIZES, max_batch=256, seed=seed, power_gain=power_gain)
    torch.cuda.synchronize()
    t0 = time.time()
    loss = ens.fit(X[tr], Y[tr], steps=train_steps, batch=128, lr=1e-3, seed=seed + 1)
    torch.cuda.synchronize()
    train_s = time.time() - t0

    def errors(sl):
        mean, _, spread = ens.answer(X[sl])
        P = Ensemble.power(Y[sl])
        return (spread, np.abs(Ensemble.power(mean) - P) / P,
                np.abs(mean[:, -1] / Y[sl][:, -1] - 1.0))

    sv, ev, _ = errors(va)
    tau = Ensemble.calibrate(sv, ev, target=target, margin=margin)
    st, et, ft = errors(te)
    return dict(rows=rows, Y=Y, records=rec, ensemble=ens, threshold=tau, spread=st,
                power_err=et, freq_err=ft, answered=st <= tau, loss=loss,
                sim_seconds=sim_s, train_seconds=train_s, runs=total)
