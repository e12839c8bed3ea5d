"""Benchmark of the per-step PIC particle loop on the single backward-wave-oscillator
workload: rippled slow-wave structure, ~200k triangles, 16M beam particles, FP32 with
fixed-point positions and currents.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step is one full cycle of the method (B update, gather + Boris + walk + scatter,
SPAI E update, re-sort every 16 steps).  Prints one JSON line (rank 0).  Under torchrun
each rank runs an independent replica of the workload (the method's state does not
shard without a domain decomposition): weak scaling, no collective on the data path.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads.bwo import EPS0, MU0, C0, QE, ME, DT_BWO, bwo_edge_field  # noqa: E402
METRIC = "particle-steps/s (gather+Boris+locate+scatter), batched runs/h vs plain, 1 GB300"
BYTES_PER_PARTICLE = 48          # particle kernel: 24 B of state read + 24 B written
CPU_SAMPLE = 160_000             # particles in the oracle's bounded sample
PUSH_PROFILE = os.path.join(ROOT, "profiles", "k_push_bwo16m.txt")


def workload(n_particles, seed=2002):
    """The single-BWO workload (workloads/bwo.py): ~200k triangles, annular 400 kV / 3 kA
    beam of n_particles macro-particles, B_z = 2.5 T, seeded small random E."""
    from workloads.bwo import bwo_workload
    return bwo_workload(n_particles, seed=seed)


def clock_sampler():
    """nvidia-smi sampled every 200 ms while the timed region runs."""
    q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")
    dev = os.environ.get("LOCAL_RANK", "0")
    try:
        p = subprocess.Popen(["nvidia-smi", "-i", dev, "--query-gpu=" + q,
                              "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None, None
    rows = []

    def reader():
        for line in p.stdout:
            rows.append(line.strip())
    t = threading.Thread(target=reader, daemon=True)
    t.start()
    return p, rows


def clock_summary(p, rows):
    if p is None:
        return None
    p.terminate()
    try:
        p.wait(timeout=5)
    except subprocess.TimeoutExpired:
        p.kill()
    time.sleep(0.1)
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for r in rows:
        f = [x.strip() for x in r.split(",")]
        if len(f) < 7:
            continue
        try:
            sm.append(float(f[0]))
            mx.append(float(f[1]))
        except ValueError:
            continue
        for name, v in zip(names, f[3:7]):
            if v.lower().startswith("active"):
                reasons.add(name)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


class NvmlClocks:
    """SM clock and clock-event (throttle) reasons of this process's GPU, read through NVML
    (libnvidia-ml, read-only queries) once before the timed region, every 2 ms by a thread
    while it runs, and once after it: a region of a few milliseconds still gets samples."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device=0):
        import ctypes
        self.ok = False
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return
            self.lib, self.ct = lib, ctypes
            h = ctypes.c_void_p()
            bus = None
            try:
                import torch
                pr = torch.cuda.get_device_properties(torch_device)
                bus = "%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
            except Exception:
                bus = None
            if bus is None or lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) != 0:
                if lib.nvmlDeviceGetHandleByIndex_v2(int(os.environ.get("LOCAL_RANK", "0")),
                                                     ctypes.byref(h)) != 0:
                    return
            self.h = h
            mx = ctypes.c_uint()
            lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))   # NVML_CLOCK_SM
            self.max_mhz = float(mx.value)
            self.ok = True
        except (OSError, AttributeError):
            self.ok = False

    def read(self):
        c = self.ct.c_uint()
        r = self.ct.c_ulonglong()
        self.lib.nvmlDeviceGetClockInfo(self.h, 1, self.ct.byref(c))
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        fn(self.h, self.ct.byref(r))
        return float(c.value), int(r.value)

    def start(self):
        self.samples = [self.read()] if self.ok else []
        self._stop = threading.Event()
        if self.ok:
            def poll():
                while not self._stop.wait(0.002):
                    self.samples.append(self.read())
            self._t = threading.Thread(target=poll, daemon=True)
            self._t.start()

    def stop(self):
        if not self.ok:
            return None
        self._stop.set()
        self._t.join()
        self.samples.append(self.read())
        reasons = set()
        for _, bits in self.samples:
            for b, name in self.REASONS.items():
                if bits & b:
                    reasons.add(name)
        return {"sm_mhz": statistics.median(m for m, _ in self.samples), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(self.samples),
                "sm_mhz_min": min(m for m, _ in self.samples), "source": "nvml"}


FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def measured_peak(key="hbm_gbs"):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_PEAKS[key], "fallback"


def push_traffic():
    """DRAM bytes per particle-kernel launch from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    try:
        src = open(os.path.join(ROOT, "paper_1701_03784_gb300", "csrc", "k_push_f32.cu"), "rb").read()
        h = hashlib.sha256(src).hexdigest()[:16]
        vals = {}
        for line in open(PUSH_PROFILE):
            if ": " in line:
                k, v = line.split(": ", 1)
                vals[k.strip()] = v.strip()
        if vals.get("k_push_f32.cu sha256[:16]") == h:
            return float(vals["dram bytes per launch (full size)"])
    except (OSError, KeyError, ValueError):
        pass
    return None


class OracleSample:
    """The FP64 oracle's particle loop (gather, Boris, walk, scatter), single-threaded, on
    a bounded sample of the same workload: the same mesh, fields and step, the first
    n_sample beam particles."""

    def __init__(self, wl, n_sample=CPU_SAMPLE, pusher="boris", threads=False):
        from oracle.operators import Mesh
        from oracle import particles as OP
        import workloads as W
        self.OP = OP
        m = Mesh(wl["nodes"], wl["tris"], wl["be"], wl["bt"])
        self.pm = OP.PushMesh(m)
        self.E = bwo_edge_field(m.N1, wl["e_scale"], 7)
        self.E[m.edge_tag == 1] = 0.0
        self.Bavg = np.zeros(m.N2)
        sl = slice(0, n_sample)
        tri, lam = OP.locate(m, wl["z"][sl], wl["r"][sl])
        self.tri = np.ascontiguousarray(tri)
        self.lam = np.ascontiguousarray(lam)
        self.u = np.ascontiguousarray(np.stack([wl["ur"][sl], wl["up"][sl], wl["uz"][sl]], 1))
        self.J, self.Q, self.Qa = np.zeros(m.N1), np.zeros(m.N0), np.zeros(m.N0)
        self.wl = wl
        self.n = n_sample
        self.n_edges = m.N1
        self.q_src = wl["weight"] * QE / (2 * math.pi)
        self.pusher = OP.VAY if pusher == "vay" else OP.BORIS
        self.threads = threads

    def step(self):
        """One particle step of the sample; returns (wall time in seconds, particles
        pushed: the live ones at the start of the step)."""
        live = int(np.count_nonzero(self.tri >= 0))
        t0 = time.perf_counter()
        self.J[:] = 0
        self.Q[:] = 0
        self.OP.push(self.pm, self.E, self.Bavg, self.wl["bz"], self.wl["dt"], QE / ME, C0,
                     self.q_src, self.tri, self.lam, self.u, self.J, self.Q, self.Qa,
                     pusher=self.pusher, threads=self.threads)
        return time.perf_counter() - t0, live


CPU_SAMPLE_THREADS = 1_600_000   # the OpenMP run's sample: enough particles per thread


def _time_sample(s, budget_s):
    done, el, pushed = 0, 0.0, 0
    while el < budget_s:
        dt_s, n = s.step()
        el += dt_s
        pushed += n
        done += 1
    return pushed / el, done


def cpu_baseline(wl, budget_s=8.0, pusher="boris"):
    """The oracle's particle loop on the host: the same particles.c built with OpenMP (all
    host cores, atomic accumulators) on a 1.6M-particle sample, and the plain
    single-threaded build on a 160k sample, each for about budget_s seconds."""
    from oracle import particles as OP
    single, n1 = _time_sample(OracleSample(wl, CPU_SAMPLE, pusher), budget_s)
    out = {"unit": "particle-steps/s", "kind": "oracle", "single_thread": single}
    try:
        threads = OP.host_threads(True)
        s = OracleSample(wl, CPU_SAMPLE_THREADS, pusher, threads=True)
        multi, nm = _time_sample(s, budget_s)
        out.update(value=multi, cores=threads, sample=(
            "FP64 C oracle particle loop (gather, %s, walk, scatter), same mesh, fields and dt: "
            "OpenMP build on %d host threads (nproc %d), the first %d of %d beam particles, "
            "%d steps; single-thread build (single_thread) on the first %d, %d steps"
            % (pusher.capitalize(), threads, os.cpu_count() or 0, CPU_SAMPLE_THREADS,
               len(wl["z"]), nm, CPU_SAMPLE, n1)))
    except RuntimeError:
        out.update(value=single, cores=1, sample=(
            "FP64 C oracle particle loop, single thread (no OpenMP compiler), the first %d of "
            "%d beam particles, %d steps" % (CPU_SAMPLE, len(wl["z"]), n1)))
    return out


def reduce_over_ranks(ms, e2e_ms, n_particles, n_slots, dist=None, device="cpu"):
    """Whole-job figures of a weak-scaling run: the slowest rank's timed regions and the
    work of all ranks (each rank advances its own replica)."""
    import torch
    t = torch.tensor([ms, e2e_ms], dtype=torch.float64, device=device)
    c = torch.tensor([float(n_particles), float(n_slots)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return t.tolist(), c.tolist()


def run_config(args, n_tris, n_edges, dt, sort_interval=None):
    """The workload named in both arms' JSON lines (sort_interval: the one in force during
    the timed steps, after the autotuner)."""
    return {"workload": "single BWO (rippled SWS, 12 periods), %d triangles, %d particles, "
                        "FP32 + int64 fixed-point J/Q" % (n_tris, args.particles),
            "n_tris": n_tris, "n_edges": n_edges, "particles": args.particles, "dt_s": dt,
            "sort_interval": args.sort_interval if sort_interval is None else sort_interval,
            "pusher": args.pusher,
            "l2": "inputs larger than L2 (particle state %d MB)" % (args.particles * 24 // 2 ** 20),
            "parallelism": "replicas" if args.gpus > 1 else "single"}


def run_reference(args):
    """The reference arm: the FP64 oracle's particle loop (the OpenMP build, on all host
    cores; the plain build if the compiler has no OpenMP), each step a bounded sample of
    the workload (its first 1.6M beam particles), rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import particles as OP
    wl = workload(args.particles)
    wl["dt"] = args.dt or DT_BWO
    try:
        cores = OP.host_threads(True)
        s = OracleSample(wl, CPU_SAMPLE_THREADS, pusher=args.pusher, threads=True)
    except RuntimeError:
        cores = 1
        s = OracleSample(wl, CPU_SAMPLE, pusher=args.pusher)
    t, pushed = 0.0, 0
    for i in range(args.warmup + args.steps):
        el, n = s.step()
        if i >= args.warmup:
            t += el
            pushed += n
    value = pushed / t
    cb = {"value": value, "unit": "particle-steps/s", "cores": cores, "kind": "oracle",
          "sample": "the first %d of %d particles per step (bounded sample of the workload), "
                    "FP64 C oracle particle loop on %d host threads (nproc %d)"
                    % (s.n, args.particles, cores, os.cpu_count() or 0)}
    line = {"metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": run_config(args, len(wl["tris"]), s.n_edges, wl["dt"]),
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


SWEEP_RUN_STEPS = 100_000   # one run of an instance: the single-BWO configuration's length


def sweep_measure(n_inst, steps, warmup, sort_interval=16, tune=True, graph=True, rank=0,
                  world=1, dist=None):
    """Batched ripple sweep: the union of n_inst seeded BWO instances (seeds 0..n_inst-1)
    advanced as one simulation (one particle-kernel launch per step over every instance)
    against the same instances run one after another, each as its own simulation, over
    the same steps and time step (0.5 x the union's stable step, i.e. the smallest
    instance limit).  Across ranks the instances are sharded (one union per rank, nothing
    exchanged) and the job's time is the slowest rank's.  Runs per hour are for runs of
    SWEEP_RUN_STEPS steps."""
    import torch
    from paper_1701_03784_gb300 import pic
    from paper_1701_03784_gb300.batch import partition
    from workloads.sweep import sweep_instance, sweep_params, sweep_particles, union, WEIGHT
    from workloads.bwo import BZ_BWO
    t_setup = time.time()
    work = [sweep_particles(i) + sweep_params(i)["n_tri"] for i in range(n_inst)]
    mine = partition(work, world)[rank]
    ins = [sweep_instance(i) for i in mine]
    u = union(ins)

    def make(x):
        mesh = pic.pic_mesh_create(x["nodes"], x["tris"], x["be"], x["bt"], eps0=EPS0, mu0=MU0,
                                   c=C0, precision=pic.PIC_FP32)
        return mesh, pic.pic_spai_build(mesh, 2, 1e-4)

    mesh_u, dt_u = make(u)
    dt = 0.5 * dt_u
    stream = torch.cuda.current_stream()
    tuned = []

    def timed(mesh, x):
        info = pic.pic_mesh_info(mesh)
        sim = pic.pic_sim_create(mesh, dt, BZ_BWO, len(x["z"]) + 1024)
        pic.pic_sim_set_sort_interval(sim, sort_interval)
        pic.pic_sim_set_graph(sim, graph)
        pic.pic_fields_set(sim, np.zeros(info["n_edges"]), np.zeros(info["n_tris"]))
        pic.pic_particles_inject(sim, x["z"], x["r"], x["ur"], x["up"], x["uz"], QE, ME, WEIGHT)
        tuned.append(pic.pic_sim_autotune(sim, 16) if tune else None)
        pic.pic_step(sim, warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pic.pic_step(sim, steps)
        e1.record(stream)
        torch.cuda.synchronize()
        d = pic.pic_diagnostics(sim)
        pic.pic_sim_destroy(sim)
        return e0.elapsed_time(e1), d

    setup_s = time.time() - t_setup
    ms_b, d_b = timed(mesh_u, u)
    ms_p = 0.0
    for x in ins:
        mesh, _ = make(x)
        ms, _ = timed(mesh, x)
        ms_p += ms
        del mesh
    (ms_b, ms_p), (n_part, n_tris) = reduce_over_ranks(ms_b, ms_p, len(u["z"]), len(u["tris"]),
                                                        dist, device="cuda")
    step_b, step_p = ms_b / steps, ms_p / steps
    runs_b = n_inst * 3600.0 / (SWEEP_RUN_STEPS * step_b * 1e-3)
    runs_p = n_inst * 3600.0 / (SWEEP_RUN_STEPS * step_p * 1e-3)
    return {"runs_per_hour": {"batched": runs_b, "plain": runs_p}, "speedup": runs_b / runs_p,
            "instances": n_inst, "seeds": "0..%d" % (n_inst - 1), "triangles": int(n_tris),
            "particles": int(n_part), "dt_s": dt,
            "dt_rule": "common step: 0.5 x the union's SPAI-stable step (the smallest instance "
                       "limit), the same in both modes",
            "timed_steps": steps, "warmup": warmup, "run_steps": SWEEP_RUN_STEPS,
            "runs_per_hour_rule": "instances x 3600 s / (run_steps x timed ms per step)",
            "cuda_graph": graph, "tuned_batched": tuned[0], "sort_interval_requested": sort_interval,
            "ms_per_step": {"batched": step_b, "plain_sum": step_p},
            "particle_steps_per_s": {"batched": n_part / (step_b * 1e-3),
                                     "plain": n_part / (step_p * 1e-3)},
            "checks": {"dce_nonzero_nodes": d_b["dce_nonzero"],
                       "walk_overflows": d_b["walk_overflows"],
                       "live_particles": d_b["n_particles"]},
            "setup_s": setup_s}


def run_sweep(args):
    """--sweep N: the batched-sweep measurement alone, as its own JSON line."""
    import torch
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    r = sweep_measure(args.sweep, args.sweep_steps, args.sweep_warmup, args.sort_interval,
                      not args.no_tune, not args.no_graph, rank, world, dist)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank != 0:
        return 0
    print(json.dumps({
        "metric": "batched runs/h vs plain", "value": r["runs_per_hour"]["batched"], "unit": "runs/h",
        "higher_is_better": True, "plain": r["runs_per_hour"]["plain"], "speedup": r["speedup"],
        "n_gpus": world, "scaling": "strong", "steps": args.sweep_steps, "warmup": args.sweep_warmup,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched ripple sweep, %d BWO instances (seeds %s)"
                               % (args.sweep, r["seeds"]),
                   "parallelism": "instances sharded over %d GPUs" % world if world > 1 else "single"},
        "batched": r}))
    return 0


SURR_STEPS, SURR_EVERY, SURR_DT = 16384, 8, 1.0e-13
SURR_VAL, SURR_TEST = 128, 128
def run_surrogate(args):
    """Surrogate of the sweep: the output-port power of args.surrogate training runs, 128
    validation and 128 held-out runs (batches of 64 instances, one union simulation each,
    SURR_STEPS steps: the beam's transit past the output plane and the ringing after it),
    a 5-member ensemble trained on the GPU, its answer gate calibrated on the validation
    runs (the largest member spread under which every validation error stays below 4%),
    its held-out accuracy where it answers, and its inference throughput."""
    import multiprocessing as mp
    import torch
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import pic, surrogate as S
    from workloads.sweep import WEIGHT, SURROGATE_SCALE, surrogate_instance
    n_train = args.surrogate
    pool = mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1))
    t0 = time.time()
    r = S.study(surrogate_instance, n_train, SURR_VAL, SURR_TEST, SURR_STEPS, SURR_EVERY,
                SURR_DT, QE, ME, WEIGHT, EPS0, MU0, C0, scale=SURROGATE_SCALE,
                train_steps=args.surrogate_steps, power_gain=args.surrogate_power_gain,
                pool=pool)
    # the pool's workers are gone before the timing (the tensor-core forward waits for
    # its kernel on the host each call, so host load shows in the device interval)
    pool.terminate()
    pool.join()
    data_s = time.time() - t0 - r["train_seconds"]
    if args.surrogate_save:
        np.savez(args.surrogate_save, X=S.features(r["rows"]), Y=r["Y"], params=r["rows"],
                 records=r["records"], record_dt=SURR_EVERY * SURR_DT)
    ens, tau, ok = r["ensemble"], r["threshold"], r["answered"]
    et, ft, loss, total = r["power_err"], r["freq_err"], r["loss"], r["runs"]
    pic_s, train_s = r["sim_seconds"], r["train_seconds"]
    # inference throughput: 65536 queries through all members
    q = torch.tensor(np.random.default_rng(5).uniform(-1, 1, (65536, 6)), dtype=torch.float32,
                     device="cuda")
    Yq = torch.empty((5, 65536, S.SIZES[-1]), dtype=torch.float32, device="cuda")
    flop = 5 * 65536 * 2 * sum(a * b for a, b in zip(S.SIZES[:-1], S.SIZES[1:]))
    times = {}
    for tc in (True, False):
        pic.pic_mlp_forward(ens.net, q, tensor_cores=tc, out=Yq)
        torch.cuda.synchronize()
        times["tensor_cores" if tc else "cuda_cores"] = _best_of(
            3, 10, lambda: pic.pic_mlp_forward(ens.net, q, tensor_cores=tc, out=Yq))
    peak, _ = measured_peak("bf16_tflops")
    tf = flop / (times["tensor_cores"] * 1e-3) / 1e12
    s_run = pic_s / total
    s_query = times["tensor_cores"] * 1e-3 / 65536
    print(json.dumps({
        "metric": "surrogate queries/s (5-member ensemble)", "value": 65536 / (times["tensor_cores"] * 1e-3),
        "unit": "queries/s", "higher_is_better": True, "n_gpus": 1, "dtype": "bf16",
        "data": "synthetic",
        "config": {"workload": "ripple-sweep surrogate: %d training, %d validation, %d held-out batched "
                               "PIC runs (%d steps = %.2f ns, dt %.3g s, coarse meshes, 5%% of the "
                               "particles); outputs: output-port power envelope (32 window means, MW; the "
                               "gate and the errors are on the arrival power, the mean of the first 12) "
                               "and the ringing frequency of the port power (4-100 GHz); instances at 450 "
                               "triangles per cm^2, their port 4.93 mm inside the output end"
                               % (n_train, SURR_VAL, SURR_TEST, SURR_STEPS, SURR_STEPS * SURR_DT * 1e9, SURR_DT),
                   "network": "5 x (6 -> 4 x 256 tanh-GELU -> 33)", "train_steps": args.surrogate_steps,
                   "batch": 128},
        "inference_ms_65536": times, "roofline": {"bound": "tensor", "achieved": tf, "peak": peak,
                                                  "unit": "TFLOP/s", "frac": tf / peak if peak else None,
                                                  "flop_per_launch": flop},
        "gate": {"spread_threshold": tau, "rule": "largest member spread (std/|mean| of the arrival "
                 "power) under which every validation error is below 4%"},
        "heldout": {"answered": float(ok.mean()),
                    "power_err_answered_max": float(et[ok].max()) if ok.any() else None,
                    "power_err_answered_median": float(np.median(et[ok])) if ok.any() else None,
                    "within_5pct_where_answered": float((et[ok] <= 0.05).mean()) if ok.any() else None,
                    "power_err_all_median": float(np.median(et)),
                    "freq_err_answered_median": float(np.median(ft[ok])) if ok.any() else None},
        "gain": {"pic_s_per_run": s_run, "surrogate_s_per_query": s_query,
                 "answers_per_s_vs_runs_per_s": s_run / s_query,
                 "effective_speedup": 1.0 / ((1.0 - ok.mean()) + ok.mean() * s_query / s_run)},
        "train_loss_last": [float(v) for v in loss],
        "seconds": {"data_total": data_s, "pic_batches": pic_s, "train": train_s}}))
    return 0


def _best_of(trials, reps, launch):
    """Milliseconds per launch: the best of `trials` CUDA-event intervals over `reps`
    launches each."""
    import torch
    best = float("inf")
    for _ in range(trials):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            launch()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / reps)
    return best


def run_mlp_queries(args):
    """Inference of a 5-member ensemble (random parameters, the surrogate's widths) on
    args.mlp_queries rows: tensor cores and CUDA cores, CUDA events, the best of 3 trials of
    10 launches each."""
    import torch
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import pic, surrogate as S
    ens = S.Ensemble(5, S.SIZES, max_batch=256, seed=9)
    n = args.mlp_queries
    q = torch.tensor(np.random.default_rng(5).uniform(-1, 1, (n, 6)), dtype=torch.float32,
                     device="cuda")
    Y = torch.empty((5, n, S.SIZES[-1]), dtype=torch.float32, device="cuda")
    flop = 5 * n * 2 * sum(a * b for a, b in zip(S.SIZES[:-1], S.SIZES[1:]))
    ms = {}
    for tc in (True, False):
        pic.pic_mlp_forward(ens.net, q, tensor_cores=tc, out=Y)
        torch.cuda.synchronize()
        ms["tensor_cores" if tc else "cuda_cores"] = _best_of(
            3, 10, lambda: pic.pic_mlp_forward(ens.net, q, tensor_cores=tc, out=Y))
    peak, kind = measured_peak("bf16_tflops")
    tf = flop / (ms["tensor_cores"] * 1e-3) / 1e12
    # training: Adam steps on minibatches of 128 with the products on either path
    Xt = torch.tensor(np.random.default_rng(6).uniform(-1, 1, (4096, 6)), dtype=torch.float32,
                      device="cuda")
    Tt = torch.tensor(np.random.default_rng(7).normal(0, 1, (4096, S.SIZES[-1])),
                      dtype=torch.float32, device="cuda")
    train_ms = {}
    for batch in (128, 256):
        for tc in (False, True):
            pic.pic_mlp_set_training(ens.net, tc)
            pic.pic_mlp_train(ens.net, Xt, Tt, batch=batch, steps=20, lr=1e-4, seed=1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pic.pic_mlp_train(ens.net, Xt, Tt, batch=batch, steps=500, lr=1e-4, seed=2)
            torch.cuda.synchronize()
            key = "batch%d_%s" % (batch, "tensor_cores" if tc else "cuda_cores")
            train_ms[key] = (time.perf_counter() - t0) / 500 * 1e3
    pic.pic_mlp_set_training(ens.net, False)
    print(json.dumps({"metric": "surrogate queries/s (5-member ensemble)",
                      "value": n / (ms["tensor_cores"] * 1e-3), "unit": "queries/s",
                      "ms": ms, "roofline": {"bound": "tensor", "achieved": tf, "peak": peak,
                                             "unit": "TFLOP/s", "frac": tf / peak,
                                             "peak_kind": kind, "flop_per_launch": flop},
                      "train_ms_per_step": train_ms}))
    return 0


SPAI_SWEEP = [(1, 1e-4), (2, 1e-2), (2, 1e-4), (3, 1e-3), (3, 1e-4)]


def _dominant_frequency(t, a, w_main, w_other):
    """Least-squares fit of two sinusoids to a(t); the frequency of the larger one."""
    from scipy.optimize import least_squares

    def res(p):
        return (p[0] * np.cos(p[2] * t) + p[1] * np.sin(p[2] * t)
                + p[3] * np.cos(p[5] * t) + p[4] * np.sin(p[5] * t) - a)
    p = least_squares(res, [a[0], 0.0, w_main, 0.0, 0.0, w_other], x_scale="jac").x
    return p[2] if np.hypot(p[0], p[1]) > np.hypot(p[3], p[4]) else p[5]


def run_spai_sweep(args):
    """SPAI pattern level and drop tolerance (Sec. 3.1 gives neither) against accuracy and
    cost.  Accuracy: the normalised cavity (c = 1, about 2000 triangles, FP64 build), TM010 +
    TM011 line integrals as E^0, 1000 steps at half the stable step; the frequencies of the
    two mode projections against the Bessel-zero closed form.  Cost: the BWO mesh (FP32
    build, no particles), the three field kernels per step, CUDA events over 2000 steps."""
    import torch
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import pic
    import workloads as W
    cav = W.cavity_mesh()
    wl = workload(1024)
    w010, w011 = W.tm0np_omega(0.5, 1.0, 1, 0), W.tm0np_omega(0.5, 1.0, 1, 1)
    rows = []
    for level, tau in SPAI_SWEEP:
        mesh = pic.pic_mesh_create(*cav, precision=pic.PIC_FP64)
        edges = pic.pic_mesh_edges(mesh)
        P0 = W.tm0np_edge_dofs(cav[0], edges, 0.5, 1.0, 1, 0)
        P1 = W.tm0np_edge_dofs(cav[0], edges, 0.5, 1.0, 1, 1)
        dt_max = pic.pic_spai_build(mesh, level, tau)
        info = pic.pic_spai_info(mesh)
        n_free = pic.pic_mesh_info(mesh)["n_free_edges"]
        dt = 0.5 * dt_max
        sim = pic.pic_sim_create(mesh, dt, 0.0, 16)
        pic.pic_fields_set(sim, P0 + P1, np.zeros(len(cav[1])))
        a0, a1 = np.zeros(1000), np.zeros(1000)
        for k in range(1000):
            E, _ = pic.pic_fields_get(sim)
            a0[k], a1[k] = E @ P0, E @ P1
            pic.pic_step(sim, 1)
        t = np.arange(1000) * dt
        f0 = _dominant_frequency(t, a0, w010, w011)
        f1 = _dominant_frequency(t, a1, w011, w010)
        pic.pic_sim_destroy(sim)
        pic.pic_mesh_destroy(mesh)

        bm = pic.pic_mesh_create(wl["nodes"], wl["tris"], wl["be"], wl["bt"], eps0=EPS0,
                                 mu0=MU0, c=C0, precision=pic.PIC_FP32)
        bdt = pic.pic_spai_build(bm, level, tau)
        binfo = pic.pic_spai_info(bm)
        bfree = pic.pic_mesh_info(bm)["n_free_edges"]
        bs = pic.pic_sim_create(bm, 0.5 * bdt, wl["bz"], 16)
        pic.pic_sim_set_graph(bs, True)
        pic.pic_fields_set(bs, bwo_edge_field(pic.pic_mesh_info(bm)["n_edges"], wl["e_scale"], 7),
                           np.zeros(len(wl["tris"])))
        pic.pic_step(bs, 100)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pic.pic_step(bs, 2000)
        e1.record()
        torch.cuda.synchronize()
        step_us = e0.elapsed_time(e1) / 2000 * 1e3
        pic.pic_sim_destroy(bs)
        pic.pic_mesh_destroy(bm)
        rows.append({"level": level, "drop_tol": tau,
                     "cavity": {"nnz_per_row": info["nnz"] / n_free,
                                "residual_rms": info["residual_rms"], "dt_stable": dt_max,
                                "tm010_rel_err": (f0 - w010) / w010,
                                "tm011_rel_err": (f1 - w011) / w011},
                     "bwo": {"nnz_per_row": binfo["nnz"] / bfree,
                             "residual_rms": binfo["residual_rms"], "dt_stable_s": bdt,
                             "field_step_us": step_us,
                             "sim_time_per_us_of_gpu": 0.5 * bdt / (step_us * 1e-6)}})
    print(json.dumps({"metric": "SPAI sweep: field-update accuracy and cost", "rows": rows,
                      "config": {"cavity": "0.5 x 1 normalised, %d triangles" % len(cav[1]),
                                 "bwo": "%d triangles, FP32, no particles" % len(wl["tris"])}}))
    return 0


def run_staircase(args):
    """Staircasing study (Sec. 5.3) on one slow-wave-structure period: the 0- and
    pi-point frequencies from cold tests on conformal and staircased meshes of the same
    spacing, against the finest conformal mesh."""
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import coldtest
    rows = []
    t0 = time.perf_counter()
    for stair in (False, True):
        for n in (500, 1000, 2000, 4000, 8000):
            f0, fpi, nt = coldtest.ring_down(n, stair)
            rows.append({"staircase": stair, "triangles": nt, "f0_GHz": f0 / 1e9,
                         "fpi_GHz": fpi / 1e9})
    ref = [r for r in rows if not r["staircase"]][-1]
    for r in rows:
        r["f0_rel_err"] = r["f0_GHz"] / ref["f0_GHz"] - 1.0
        r["fpi_rel_err"] = r["fpi_GHz"] / ref["fpi_GHz"] - 1.0
    print(json.dumps({"metric": "staircasing: cold-test frequency error of one SWS period",
                      "unit": "relative", "rows": rows,
                      "wall_s": time.perf_counter() - t0,
                      "config": {"workload": "one period (7.5 mm) of R(z) = 15 + 2.1 cos(2 pi z "
                                             "/ 7.5 mm) mm between ripple maxima, FP64, 1.5 ns "
                                             "ring-down, reference: the finest conformal mesh"}}))
    return 0


def run_diode(args):
    """Planar diode at 100 kV over 1 cm (Sec. 5.2's check on a planar gap): injection
    scan against the relativistic planar space-charge-limited current -- the fraction
    returned to the cathode (a virtual cathode) and the central current density that
    crosses the gap -- on the planar check's setup (6 cm emitter in a 7 cm tube, 5 T guide
    field, ~20k triangles graded toward the cathode, 2000 births per step, 10,000 +
    10,000 steps); then the diode configuration as stated (1 cm disk, 2 cm tube, ~20k
    uniform triangles, no guide field) over-injected, and its throughput."""
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import diode
    from oracle import sources as OS
    J_scl = OS.child_langmuir_planar(1e5, 1e-2, QE / ME, EPS0, C0)
    J_cl = diode.classical_limit(1e5, 1e-2)
    rows = []
    t0 = time.perf_counter()
    for f in (0.9, 0.95, 1.0, 1.05, 1.1, 1.3):
        r = diode.run(over=f * J_scl / J_cl)
        rows.append({"inject_over_law": f, "return_fraction": r["return_fraction"],
                     "J_center_over_law": r["J_center"] / J_scl,
                     "I_anode_over_I_emitted": r["I_anode"] / r["I_emitted"],
                     "in_flight_end": r["n_particles"], "steps": r["steps"],
                     "emit_dropped": r["emit_dropped"], "dce_nonzero": r["dce_nonzero"]})
    stated = diode.run(radius=2e-2, r_emit=1e-2, r_measure=0.3e-2, bz=0.0, grade=1.0,
                       over=1.3 * J_scl / J_cl)
    m2 = diode.throughput()
    print(json.dumps({"metric": "planar diode: space-charge limit / relativistic Child-Langmuir",
                      "unit": "ratio", "law_over_classical": J_scl / J_cl,
                      "rows": rows, "wall_s": time.perf_counter() - t0,
                      "stated_1cm_disk_over_1.3": {
                          "J_center_over_law": stated["J_center"] / J_scl,
                          "return_fraction": stated["return_fraction"],
                          "in_flight_end": stated["n_particles"],
                          "note": "a 1 cm disk 1 cm from the anode is a two-dimensional diode: "
                                  "its limit exceeds the planar law (finite-emitter enhancement)"},
                      "m2_throughput": m2,
                      "config": {"workload": "planar diode 100 kV, 1 cm gap; scan: 6 cm emitter, "
                                             "7 cm tube, 5 T, ~20k triangles graded to the "
                                             "cathode (0.35), 2000 births per step, FP32, "
                                             "10000 + 10000 steps per injection"}}))
    return 0


M2_SETTLE = 4000


def measure_m2():
    """The diode configuration as stated (1 cm disk, 1 cm gap, 100 kV, ~20k triangles,
    2000 births per step) once its gap has filled: throughput at that particle count."""
    from paper_1701_03784_gb300 import diode
    r = diode.throughput(settle_steps=M2_SETTLE)
    r["workload"] = ("diode: 1 cm cathode disk, 1 cm gap, 100 kV, 2 cm tube, %d triangles, "
                     "%d births per step at rest, FP32; timed after %d steps"
                     % (r["n_tris"], r["births_per_step"], M2_SETTLE))
    r["value"] = r.pop("particle_steps_per_s")
    r["unit"] = "particle-steps/s"
    return r


def _timed_steps(pic, sim, steps):
    """(ms per step, ms per particle-kernel launch) over `steps` steps, CUDA events."""
    import torch
    torch.cuda.synchronize()
    pic.pic_kernel_timing(sim, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    pic.pic_step(sim, steps)
    e1.record()
    torch.cuda.synchronize()
    push_ms, n = pic.pic_kernel_timing(sim, False)
    return e0.elapsed_time(e1) / steps, push_ms / max(n, 1)


def measure_m3u(pic, mesh, wl, dt, peak, per_tri=100, steps=200, warmup=20):
    """The same mesh with about per_tri particles per triangle spread uniformly (in area)
    over the whole domain, momenta of the beam (400 kV drift along z, thermal 1e-3 u_z):
    the contention-free counterpart of the beam workload.  FP32 build."""
    import workloads as W
    n_tris = len(wl["tris"])
    n = per_tri * n_tris
    uz0 = float(np.median(wl["uz"]))
    z, r, ur, up, uz = W.uniform_in_mesh(wl["nodes"], wl["tris"], n, 2013, sigma_u=1e-3 * uz0,
                                         drift=(0.0, 0.0, uz0))
    info = pic.pic_mesh_info(mesh)
    sim = pic.pic_sim_create(mesh, dt, wl["bz"], n + 1024)
    pic.pic_fields_set(sim, bwo_edge_field(info["n_edges"], wl["e_scale"], 7), np.zeros(n_tris))
    pic.pic_particles_inject(sim, z, r, ur, up, uz, QE, ME, wl["weight"])
    pic.pic_step(sim, warmup)
    live0 = pic.pic_diagnostics(sim)["n_particles"]
    step_ms, push_ms = _timed_steps(pic, sim, steps)
    live1 = pic.pic_diagnostics(sim)["n_particles"]
    pic.pic_sim_destroy(sim)
    avg = 0.5 * (live0 + live1)
    gbs = BYTES_PER_PARTICLE * avg / (push_ms * 1e-3) / 1e9
    return {"workload": "same mesh, %d particles uniform over all %d triangles (%d per "
                        "triangle), beam momenta, FP32" % (n, n_tris, per_tri),
            "value": avg / (step_ms * 1e-3), "unit": "particle-steps/s", "steps": steps,
            "warmup": warmup, "ms_per_step": step_ms, "push_ms": push_ms,
            "push_gbs": gbs, "push_frac_of_hbm": gbs / peak, "live_particles": [live0, live1]}


BYTES_PER_PARTICLE_FP64 = 88   # FP64 build: 44 B of state read + 44 B written


def measure_fp64(pic, wl, dt, peak, steps=200, warmup=20):
    """The beam workload in the FP64 build (the paper's arithmetic): FP64 fields, particle
    state and currents, the same mesh, particles and step."""
    mesh = pic.pic_mesh_create(wl["nodes"], wl["tris"], wl["be"], wl["bt"], eps0=EPS0, mu0=MU0,
                               c=C0, precision=pic.PIC_FP64)
    pic.pic_spai_build(mesh, 2, 1e-4)
    info = pic.pic_mesh_info(mesh)
    n = len(wl["z"])
    sim = pic.pic_sim_create(mesh, dt, wl["bz"], n + 1024)
    pic.pic_fields_set(sim, bwo_edge_field(info["n_edges"], wl["e_scale"], 7),
                       np.zeros(info["n_tris"]))
    pic.pic_particles_inject(sim, wl["z"], wl["r"], wl["ur"], wl["up"], wl["uz"], QE, ME,
                             wl["weight"])
    pic.pic_step(sim, warmup)
    live0 = pic.pic_diagnostics(sim)["n_particles"]
    step_ms, push_ms = _timed_steps(pic, sim, steps)
    d = pic.pic_diagnostics(sim)
    pic.pic_sim_destroy(sim)
    pic.pic_mesh_destroy(mesh)
    avg = 0.5 * (live0 + d["n_particles"])
    gbs = BYTES_PER_PARTICLE_FP64 * avg / (push_ms * 1e-3) / 1e9
    return {"workload": "single BWO, %d particles, FP64 build" % n, "dtype": "f64",
            "value": avg / (step_ms * 1e-3), "unit": "particle-steps/s", "steps": steps,
            "warmup": warmup, "ms_per_step": step_ms, "push_ms": push_ms,
            "bytes_per_particle": BYTES_PER_PARTICLE_FP64, "push_gbs": gbs,
            "push_frac_of_hbm": gbs / peak, "dce_max": d["dce_max"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--particles", type=int, default=16_000_000)
    ap.add_argument("--sort-interval", type=int, default=16)
    ap.add_argument("--dt", type=float, default=None)
    ap.add_argument("--pusher", default="boris", choices=["boris", "vay"],
                    help="velocity update of Eq. DLE (both arms)")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra records (uniform-fill M3u, FP64 build, batched sweep)")
    ap.add_argument("--batched", type=int, default=16,
                    help="instances of the batched-sweep record in the default line (0: none)")
    ap.add_argument("--sweep", type=int, default=0,
                    help="batched ripple sweep over this many instances instead")
    ap.add_argument("--sweep-steps", type=int, default=64)
    ap.add_argument("--sweep-warmup", type=int, default=16)
    ap.add_argument("--surrogate", type=int, default=0,
                    help="surrogate of the sweep trained on this many batched PIC runs instead")
    ap.add_argument("--surrogate-steps", type=int, default=8000)
    ap.add_argument("--surrogate-power-gain", type=float, default=16.0,
                    help="weight of the arrival power in the loss, as a factor on its standardised target")
    ap.add_argument("--surrogate-save", default=None,
                    help="write the surrogate's inputs and PIC outputs to this .npz")
    ap.add_argument("--mlp-queries", type=int, default=0,
                    help="time surrogate-network inference on this many queries instead")
    ap.add_argument("--spai-sweep", action="store_true",
                    help="SPAI pattern / drop-tolerance sweep (accuracy and cost) instead")
    ap.add_argument("--staircase", action="store_true",
                    help="staircasing study: cold tests of one SWS period instead")
    ap.add_argument("--diode", action="store_true",
                    help="planar space-charge-limited diode (static field + emission) instead")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the launch-shape autotuner (fixed re-sort interval and shapes)")
    ap.add_argument("--no-graph", action="store_true",
                    help="sweep: launch every step's kernels instead of replaying a CUDA graph")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep:
        return run_sweep(args)
    if args.surrogate:
        return run_surrogate(args)
    if args.mlp_queries:
        return run_mlp_queries(args)
    if args.spai_sweep:
        return run_spai_sweep(args)
    if args.diode:
        return run_diode(args)
    if args.staircase:
        return run_staircase(args)

    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import paper_1701_03784_gb300 as pkg
    pkg.build()
    from paper_1701_03784_gb300 import pic

    wl = workload(args.particles, seed=2002 + rank)
    mesh = pic.pic_mesh_create(wl["nodes"], wl["tris"], wl["be"], wl["bt"], eps0=EPS0, mu0=MU0,
                               c=C0, precision=pic.PIC_FP32)
    dt_max = pic.pic_spai_build(mesh, 2, 1e-4)
    dt = args.dt or DT_BWO
    wl["dt"] = dt
    info = pic.pic_mesh_info(mesh)
    sim = pic.pic_sim_create(mesh, dt, wl["bz"], args.particles + 1024)
    pic.pic_sim_set_sort_interval(sim, args.sort_interval)
    if args.pusher == "vay":
        pic.pic_sim_set_pusher(sim, pic.PIC_PUSHER_VAY)
    import workloads as W
    E0 = bwo_edge_field(info["n_edges"], wl["e_scale"], 7 + rank)
    pic.pic_fields_set(sim, E0, np.zeros(info["n_tris"]))
    pic.pic_particles_inject(sim, wl["z"], wl["r"], wl["ur"], wl["up"], wl["uz"], QE, ME,
                             wl["weight"])
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # launch shapes (re-sort interval, particle-kernel grid, field-kernel block), then warm-up
    tuned = None if args.no_tune else pic.pic_sim_autotune(sim, 32)
    pic.pic_step(sim, args.warmup)
    barrier()
    d0 = pic.pic_diagnostics(sim)
    n_live = d0["n_particles"]
    si = int(d0["sort_interval"])
    # phase of the re-sort: the first timed step ends with one, so the K timed steps hold
    # ceil(K / interval) re-sorts (never fewer than their amortised share)
    if si > 0:
        pic.pic_step(sim, (si - 1 - int(d0["steps_since_sort"])) % si)
    resorts = -(-args.steps // si) if si > 0 else 0
    # timed region: K full steps, CUDA events on the launching stream
    pic.pic_kernel_timing(sim, True)
    clk = NvmlClocks(local)
    sampler, rows = (None, None) if clk.ok else clock_sampler()
    barrier()
    launches0 = pic.pic_launch_count()
    clk.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    pic.pic_step(sim, args.steps)
    ev1.record(stream)
    barrier()
    ms = ev0.elapsed_time(ev1)
    clocks = clk.stop() if clk.ok else clock_summary(sampler, rows)
    launches = pic.pic_launch_count() - launches0
    push_ms, push_launches = pic.pic_kernel_timing(sim, False)
    diag = pic.pic_diagnostics(sim)
    n_end = diag["n_particles"]

    # end to end through the C ABI with host buffers: every step uploads the state from
    # pinned memory, steps and reads it back (pic_step_host)
    n_slots = pic.pic_particles_count(sim)
    bpp = pic.pic_particles_raw_bytes(sim)
    host = torch.empty(pic.pic_particles_raw_size(sim, n_slots), dtype=torch.uint8,
                       pin_memory=True)
    pic.pic_particles_raw_get(sim, host.data_ptr(), n_slots)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pic.pic_step_host(sim, host.data_ptr(), n_slots, args.e2e_steps)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)

    (ms, e2e_ms), (total_particles, total_slots) = reduce_over_ranks(
        ms, e2e_ms, 0.5 * (n_live + n_end), n_slots, dist, device="cuda")
    value = total_particles * args.steps / (ms * 1e-3)
    e2e_value = total_slots * args.e2e_steps / (e2e_ms * 1e-3)

    if rank == 0:
        peak, peak_kind = measured_peak()
        avg_push_s = push_ms * 1e-3 / max(push_launches, 1)
        achieved = BYTES_PER_PARTICLE * 0.5 * (n_live + n_end) / avg_push_s / 1e9
        traffic = push_traffic()
        line = {
            "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": run_config(args, info["n_tris"], info["n_edges"], dt, si),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_push_f32", "peak_kind": peak_kind,
                         "bytes_per_particle": BYTES_PER_PARTICLE,
                         "avg_launch_ms": avg_push_s * 1e3, "launches": push_launches},
            "e2e": {"value": e2e_value, "unit": "particle-steps/s",
                    "h2d_bytes_per_step": n_slots * bpp, "d2h_bytes_per_step": n_slots * bpp,
                    "steps": args.e2e_steps},
            "gpu_launches": launches,
            "gpu_launches_counted": "kernels the library enqueued in the timed region "
                                    "(pic_launch_count before and after)",
            "tuning": tuned,
            "resorts_in_timed_region": resorts,
            "clocks": clocks,
            "checks": {"dt_over_stable": dt / dt_max,
                       "dce_nonzero_nodes": diag["dce_nonzero"], "dgl_drift": diag["dgl_drift"],
                       "walk_overflows": diag["walk_overflows"], "live_particles": n_end,
                       "absorbed": diag["n_absorbed"]},
        }
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(wl, pusher=args.pusher)
        if not args.no_extras:
            line["m3u"] = measure_m3u(pic, mesh, wl, dt, peak)
            del mesh
            line["fp64"] = measure_fp64(pic, wl, dt, peak)
            line["m2"] = measure_m2()
            if args.batched:
                line["batched"] = sweep_measure(args.batched, 320, 32)
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
