"""Benchmark of the Ising-film sweep on GB300: spin-flip attempts per ns.

One step = 10 checkerboard Metropolis sweeps of the 120 x 240 x 1600 film
(46,080,000 spins, Eq. 11 boundary, H1 = +0.55, T = 3) plus one record of the
int64 sums B, M, M1, Mn, m(kx) -- the film and cadence of the paper-scale run.
The default run times 200 steps (the 2000 sweeps of that run) after 3 warm-up
steps, flushing L2 between steps, and prints one JSON line with the roofline
of the update kernel, the oracle's CPU rate, an end-to-end figure through
host buffers, clocks, and bounded batched/serving runs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun every rank runs its own replica of the film (independent
chains, no collective: weak scaling); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

def alu_frac(attempts_per_ns):
    """Fraction of the update kernels' ALU roofline (OPS_PER_ATTEMPT int32 ops
    per attempt against 152 SMs x 128 lanes x 2.07 GHz)."""
    return attempts_per_ns * OPS_PER_ATTEMPT / (N_SM * LANES_PER_SM * SM_MAX_GHZ)


SHAPE_NAMES = {0: "auto", 1: "resident", 2: "grid, 1 word/thread", 3: "grid, 2 words/thread",
               4: "grid, 4 threads/word", 5: "cluster-resident"}
SHAPE_FLAGS = {1: "resident", 2: "grid1", 3: "grid2", 4: "gridq", 5: "cluster"}
METRIC = "spin-flip attempts/ns on 1 GB300, batched vs plain, % roofline; p99 latency"
UNIT = "attempts/ns"
SWEEPS_PER_STEP = 10
# Algorithmic integer work per attempt: Philox4x32-10 shared by 4 sites
# (10 rounds x (2 mul-hi + 2 mul-lo + 4 xor) + 9 x 2 key adds = 98 ops) = 24.5,
# plus neighbour count (1), threshold select/compare (3), flip (1): 29.5 -> 30.
OPS_PER_ATTEMPT = 30
# INT32 peak: 152 SMs x 4 schedulers x 32 lanes (one warp instruction per
# scheduler per cycle) x 2.07 GHz maximum SM clock.
N_SM, LANES_PER_SM, SM_MAX_GHZ = 152, 128, 2.07
PROFILE = os.path.join(ROOT, "profiles", "update_film_kernel_film46m.md")
KERNEL_SOURCES = ["paper_1411_5588_gb300/csrc/ising_kernels.cu", "paper_1411_5588_gb300/csrc/ising_device.cuh",
                  "paper_1411_5588_gb300/csrc/ising_launch.h"]


def kernel_source_hash():
    h = hashlib.sha1()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(shape):
    """dram bytes per update launch from the committed ncu summary, if it was
    taken on the current kernel source in the launch shape this run used."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    m = re.search(r"kernel-source-sha1:\s*([0-9a-f]{40})", text)
    t = re.search(r"dram-bytes-per-launch:\s*([0-9.eE+]+)", text)
    s = re.search(r"launch-shape:\s*(\S+)", text)
    if not m or not t or not s or m.group(1) != kernel_source_hash() or s.group(1) != SHAPE_FLAGS[shape]:
        return None
    return float(t.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = str(gpu_index)
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", self.gpu], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, device="cpu"):
    """Maximum of a float over all ranks of the default process group (the
    value itself when no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def cpu_baseline(min_seconds=10.0, max_sweeps=40):
    """The oracle, as it stands, on the host cores: sweeps of the 46M-site
    film after its slab start, until about min_seconds of CPU work."""
    from oracle import oracle as O
    from paper_1411_5588_gb300 import workloads as WL
    job = WL.film_46m()
    ncores = os.cpu_count() or 1
    O.set_threads(ncores)
    f = O.Film(job["Lx"], job["Ly"], job["Lz"], job["J"], job["H1"], job["T"], job["seed"])
    f.init(O.INIT_SLAB_Y, job["flip_p"])
    t0 = time.perf_counter()
    n = 0
    while n < max_sweeps and (n == 0 or time.perf_counter() - t0 < min_seconds):
        f.sweep(1, 0)
        n += 1
    dt = time.perf_counter() - t0
    att = WL.sites(job) * n
    cores = O.get_threads()
    # the same oracle on one core, continuing the chain (two sweeps)
    O.set_threads(1)
    t1 = time.perf_counter()
    for _ in range(2):
        f.sweep(1, 0)
    d1 = time.perf_counter() - t1
    O.set_threads(ncores)
    a1 = WL.sites(job) * 2
    return {"value": att / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} sweeps of the 120x240x1600 film after its slab start ({att} attempts, {dt:.1f} s)",
            "single_core": {"value": a1 / d1 / 1e9, "unit": UNIT, "cores": 1,
                            "sample": f"the next 2 sweeps on one thread ({a1} attempts, {d1:.1f} s)"}}


def reference_arm(args):
    """--impl reference: the CPU oracle on the host cores, one sweep of the
    46M-site film per step with a record after every 10th sweep: the timed
    workload's mix of sweeps and records, in steps a tenth as long."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1411_5588_gb300 import workloads as WL
    job = WL.film_46m()
    O.set_threads(os.cpu_count() or 1)
    f = O.Film(job["Lx"], job["Ly"], job["Lz"], job["J"], job["H1"], job["T"], job["seed"])
    f.init(O.INIT_SLAB_Y, job["flip_p"])
    for _ in range(args.warmup):
        f.sweep(1, 0)
    t0 = time.perf_counter()
    for i in range(args.steps):
        f.sweep(1, 0)
        if (i + 1) % SWEEPS_PER_STEP == 0:
            f.measure()
    dt = time.perf_counter() - t0
    att = WL.sites(job) * args.steps
    value = att / dt / 1e9
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "i8", "data": "synthetic", "impl": "reference",
            "config": {"workload": "film 120x240x1600 (46,080,000 spins), Eq. 11 y boundary, H1=+0.55, T=3, "
                                   "slab start + 1% flips, seed 2; 10 sweeps + one int64 record per step, "
                                   "sampled as one sweep per step with a record every 10th sweep (CPU)",
                       "parallelism": f"openmp x{O.get_threads()}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.get_threads(), "kind": "oracle",
                             "sample": f"{args.steps} sweeps of the 120x240x1600 film, "
                                       f"{args.steps // SWEEPS_PER_STEP} record(s), one after every "
                                       f"{SWEEPS_PER_STEP}th sweep"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batched_vs_plain(ig, WL, torch, sweeps=20):
    """64-film integration set: one batch (shared launches, CUDA graph) vs the
    same films run one after another through the single-film path.  Both
    time sweeps only (creation and initial states excluded)."""
    jobs = WL.ti_batch(n_sweeps=2 * sweeps)
    for j in jobs:
        j["measure_every"] = 10
    per_sweep = sum(WL.sites(j) for j in jobs)
    b = ig.Batch(jobs)
    shape = SHAPE_NAMES[b.autotune()]
    b.reserve_records(2 * sweeps)
    b.sweep(sweeps, True)  # warm-up (captures the graph)
    b.synchronize()
    t0 = time.perf_counter()
    b.sweep(2 * sweeps, True)
    b.synchronize()
    tb = time.perf_counter() - t0
    lanes = b.lanes
    b.close()
    batched = per_sweep * 2 * sweeps / tb / 1e9
    tp = 0.0
    for j in jobs:
        g = ig.Film(j["Lx"], j["Ly"], j["Lz"], j["J"], j["H1"], j["T"], j["seed"], replica=j["replica"])
        g.init(j["init_kind"])
        g.autotune(10)
        g.synchronize()
        t0 = time.perf_counter()
        g.sweep(sweeps, 10)
        g.synchronize()
        tp += time.perf_counter() - t0
        g.read_series()
        g.close()
    plain = per_sweep * sweeps / tp / 1e9
    return {"workload": "64 films 32x64x128..96x192x384 (16 H1 nodes x 2 T x 2 seeds), records every 10 sweeps",
            "batched": batched, "plain": plain, "ratio": batched / plain, "unit": UNIT, "batched_shape": shape,
            "batched_lanes": lanes,
            "batched_alu_frac": alu_frac(batched),
            "note": "both sides autotuned (library autotuner) before timing",
            "sweeps": {"batched": 2 * sweeps, "plain_per_film": sweeps}}


def serving(ig, WL, n_jobs=2000, chunk=50, budget=16 << 30):
    """Poisson stream of jobs into the continuous-batching server."""
    jobs = WL.serve_2000(n_jobs=n_jobs)
    srv = ig.Server(budget, chunk_sweeps=chunk)
    t0 = time.perf_counter()
    tickets = []
    for j in jobs:
        delay = j["arrival"] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        tickets += srv.submit([j])
    lat = []
    att = 0
    for t, j in zip(tickets, jobs):
        srv.wait(t, 3600.0)
        _, _, info = srv.result(t, want_spins=False)
        lat.append(info["t_finish"] - info["t_submit"])
        att += WL.sites(j) * j["n_sweeps"]
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat.sort()
    q = lambda p: lat[min(len(lat) - 1, int(math.ceil(p * len(lat))) - 1)]
    return {"workload": f"{n_jobs} jobs, Poisson 200/s, sizes 16^3..96x192x768, 500-5000 sweeps",
            "attempts_per_ns": att / wall / 1e9, "p50_latency_s": q(0.50), "p99_latency_s": q(0.99),
            "wall_s": wall, "offered_attempts_per_ns": att / (jobs[-1]["arrival"] + 1e-9) / 1e9,
            "chunk_sweeps": chunk, "chunks": st["chunks"]}


def serving_capacity(ig, WL, n_jobs=400, n_plain=40, chunk=50, budget=16 << 30):
    """Saturated server (the first n_jobs of the stream submitted at once)
    against the same kind of jobs run one after another through the
    single-film path (the first n_plain of them)."""
    jobs = WL.serve_2000()[:n_jobs]
    srv = ig.Server(budget, chunk_sweeps=chunk)
    t0 = time.perf_counter()
    tickets = srv.submit(jobs)
    for t in tickets:
        srv.wait(t, 3600.0)
        srv.result(t, want_spins=False)
    served = sum(WL.sites(j) * j["n_sweeps"] for j in jobs) / (time.perf_counter() - t0) / 1e9
    srv.close()
    att = 0
    t0 = time.perf_counter()
    for j in jobs[:n_plain]:
        g = ig.Film(j["Lx"], j["Ly"], j["Lz"], j["J"], j["H1"], j["T"], j["seed"], replica=j["replica"])
        g.init(j["init_kind"])
        g.sweep(j["n_sweeps"], j["measure_every"])
        g.read_series()
        g.get_spins()
        g.close()
        att += WL.sites(j) * j["n_sweeps"]
    plain = att / (time.perf_counter() - t0) / 1e9
    return {"workload": f"first {n_jobs} jobs of the stream submitted at once; plain: first {n_plain} one at a time "
                        "(create, initial state, sweeps, records and spins back)",
            "served": served, "plain": plain, "ratio": served / plain, "unit": UNIT}


def film_8_run(ig, WL):
    """The 8^3 film over its whole run: 10^4 sweeps, a record after each,
    on the resident kernel (the default for a film this small) and on the
    grid kernels."""
    job = WL.film_8()
    out = {"workload": "8x8x8 film, 10^4 sweeps, a record every sweep"}
    for name, shape in (("resident", ig.SHAPE_RESIDENT), ("grid", ig.SHAPE_GRID_1)):
        g = ig.Film(job["Lx"], job["Ly"], job["Lz"], job["J"], job["H1"], job["T"], job["seed"], shape=shape)
        g.init(job["init_kind"])
        g.synchronize()
        t0 = time.perf_counter()
        g.sweep(job["n_sweeps"], job["measure_every"])
        recs = g.read_series()
        dt = time.perf_counter() - t0
        g.close()
        out[name] = {"records": int(recs.shape[0]), "attempts_per_ns": WL.sites(job) * job["n_sweeps"] / dt / 1e9,
                     "wall_s": dt}
    out["attempts_per_ns"] = out["resident"]["attempts_per_ns"]
    return out


def t_scan_slice(ig, WL, sweeps=10):
    """The 40-film temperature scan (40 x 120x240x1600) as one autotuned
    batch, a few sweeps with a record after every sweep."""
    jobs = WL.t_scan_40(n_sweeps=sweeps + 1)
    b = ig.Batch(jobs)
    shape = SHAPE_NAMES[b.autotune()]
    b.reserve_records(sweeps + 1)
    b.sweep(1)
    b.synchronize()
    t0 = time.perf_counter()
    b.sweep(sweeps)
    b.synchronize()
    dt = time.perf_counter() - t0
    lanes = b.lanes
    b.close()
    a = sum(WL.sites(j) for j in jobs) * sweeps / dt / 1e9
    return {"workload": f"40 films 120x240x1600 (T = 1.5..4.4), {sweeps} sweeps with a record every sweep",
            "attempts_per_ns": a, "alu_frac": alu_frac(a), "wall_s": dt, "shape": shape, "lanes": lanes}


def procedures(ig, WL):
    """The paper's procedures at their default sizes, each film set in one
    batch. It runs the beta integration for gamma(pi/2) and tau(0, pi/2), then
    the contact angle, Young difference and gamma(theta) scan, then stiffness
    and step free energy, then the line tension over a constant-area set.
    Sweeps are timed on the device side (synchronised wall clock) and the
    host reductions separately."""
    import numpy as np

    from paper_1411_5588_gb300 import workflows as PW

    def timed_run(wl):
        b = ig.Batch(wl["jobs"])
        shape = SHAPE_NAMES[b.autotune()]
        b.reserve_records(wl["n_sweeps"])  # records every sweep: no ring growth while timed
        b.synchronize()
        t0 = time.perf_counter()
        b.sweep(wl["n_sweeps"], True)
        b.synchronize()
        dt = time.perf_counter() - t0
        recs = [b.read_series(i) for i in range(len(wl["jobs"]))]
        lanes = b.lanes
        if shape == SHAPE_NAMES[5]:
            shape += f", {b.cluster_size} CTAs per film"
        b.close()
        att = sum(WL.sites(j) for j in wl["jobs"]) * wl["n_sweeps"]
        return recs, {"films": len(wl["jobs"]), "attempts": att, "sweep_s": dt, "attempts_per_ns": att / dt / 1e9,
                      "alu_frac": alu_frac(att / dt / 1e9), "shape": shape, "lanes": lanes}

    out = {}
    it = WL.interface_tension_set()
    recs, out["interface_tension_run"] = timed_run(it)
    t0 = time.perf_counter()
    r_it = PW.interface_tension(it, recs)
    out["interface_tension"] = {"sizes": it["sizes"], "Ly": it["Ly"], "T": it["T"], "n_beta": len(it["betas"]),
                                "dF": r_it["dF"].tolist(), "gamma_pi2": r_it["gamma_pi2"], "tau0": r_it["tau0"],
                                "host_s": time.perf_counter() - t0}
    ca = WL.contact_angle_set()
    recs, out["contact_angle_run"] = timed_run(ca)
    t0 = time.perf_counter()
    r_ca = PW.contact_angle(ca, recs, r_it["gamma_pi2"])
    r_st = PW.stiffness_and_steps(r_ca["theta"], r_ca["gamma"], r_it["gamma_pi2"], ca["T"], ca["Lx"], ca["Lz"],
                                  ca["H1s"])
    out["contact_angle"] = {"film": [ca["Lx"], ca["Ly"], ca["Lz"]], "T": ca["T"], "H1": list(ca["H1s"]),
                            "theta_deg": np.degrees(r_ca["theta"]).tolist(),
                            "theta_young_deg": np.degrees(r_ca["theta_young"]).tolist(),
                            "delta_f1": r_ca["delta_f1"].tolist(), "gamma": r_ca["gamma"].tolist(),
                            "stiffness_c": r_st["c"], "kappa": r_st["kappa"], "f_s": r_st["f_s"],
                            "host_s": time.perf_counter() - t0}
    lt = WL.line_tension_set()
    j = list(ca["H1s"]).index(lt["H1"])
    recs, out["line_tension_run"] = timed_run(lt)
    t0 = time.perf_counter()
    r_lt = PW.line_tension(lt, recs, r_ca["theta"][j], r_ca["gamma"][j], r_it["gamma_pi2"])
    out["line_tension"] = {"sizes": [list(v) for v in lt["sizes"]], "H1": lt["H1"], "R": r_lt["R"].tolist(),
                           "dtau": r_lt["dtau"], "intercept": r_lt["intercept"], "host_s": time.perf_counter() - t0}
    out["physics_note"] = ("not converged: a throughput leg (2000 sweeps, 500 discarded, sizes scaled down from "
                           "the paper's); its physics values are not estimates of the paper's quantities")
    runs = [out[k] for k in ("interface_tension_run", "contact_angle_run", "line_tension_run")]
    out["attempts_per_ns"] = sum(r["attempts"] for r in runs) / sum(r["sweep_s"] for r in runs) / 1e9
    out["unit"] = UNIT
    return out


def one_field_set(ig, WL, sweeps=1000):
    """The contact-angle procedure at one surface field (10 films 32x96x64,
    a record every sweep): too few words per half-sweep to fill the GPU, the
    case the cluster-resident shape is for.  Autotuned (all shapes) against
    the faster of the grid shapes GRID_1 and GRID_Q, each pinned."""
    jobs = WL.contact_angle_set(H1s=(0.3,), n_sweeps=sweeps)["jobs"]
    att = sum(WL.sites(j) for j in jobs) * sweeps

    def timed(shape=None):
        b = ig.Batch(jobs)
        picked = SHAPE_NAMES[b.autotune()] if shape is None else SHAPE_NAMES[shape]
        if shape is not None:
            b.set_shape(shape)
        if b.get_shape() == ig.SHAPE_CLUSTER:
            picked += f", {b.cluster_size} CTAs per film"
        b.reserve_records(sweeps + 8)
        b.sweep(8, True)
        b.synchronize()
        for i in range(len(jobs)):
            b.read_series(i)
        t0 = time.perf_counter()
        b.sweep(sweeps, True)
        b.synchronize()
        dt = time.perf_counter() - t0
        b.close()
        return att / dt / 1e9, picked

    auto, shape = timed()
    grid = max(timed(ig.SHAPE_GRID_1)[0], timed(ig.SHAPE_GRID_Q)[0])
    return {"films": len(jobs), "film": [32, 96, 64], "sweeps": sweeps, "autotuned": auto, "shape": shape,
            "grid_best": grid, "ratio": auto / grid, "unit": UNIT}


PROFILE_SETS = ("ti64", "contact_angle", "interface_tension", "line_tension", "contact_angle_one_field")


def profile_set(args):
    """--profile-set: one film set as a batch for a few sweeps in a fixed
    launch shape, records after every sweep unless --profile-every says
    otherwise (0: none), in one lane unless --profile-lanes says otherwise (so
    that one launch covers the whole set).  The command the batch kernels'
    ncu summaries in profiles/ are captured from; it prints one summary line,
    not a benchmark line."""
    import paper_1411_5588_gb300 as ig
    from paper_1411_5588_gb300 import workloads as WL
    n = args.profile_sweeps
    jobs = {"ti64": lambda: WL.ti_batch(n_sweeps=n),
            "contact_angle": lambda: WL.contact_angle_set(n_sweeps=n)["jobs"],
            "interface_tension": lambda: WL.interface_tension_set(n_sweeps=n)["jobs"],
            "line_tension": lambda: WL.line_tension_set(n_sweeps=n)["jobs"],
            "contact_angle_one_field": lambda: WL.contact_angle_set(H1s=(0.3,), n_sweeps=n)["jobs"]}[args.profile_set]()
    if args.profile_every is not None:
        jobs = [dict(j, measure_every=args.profile_every) for j in jobs]
    b = ig.Batch(jobs, lanes=args.profile_lanes)
    if args.profile_shape == "cluster":
        b.set_cluster_size(args.profile_cluster)
    b.set_shape({"grid1": ig.SHAPE_GRID_1, "grid2": ig.SHAPE_GRID_2, "gridq": ig.SHAPE_GRID_Q,
                 "cluster": ig.SHAPE_CLUSTER}[args.profile_shape])
    cl = f" ({b.cluster_size} CTAs per film)" if args.profile_shape == "cluster" else ""
    if args.profile_every != 0:
        b.reserve_records(n)
    b.sweep(n, False)
    b.synchronize()
    lanes = b.lanes
    b.close()
    print(f"{args.profile_set}: {len(jobs)} films in {lanes} lane(s), {n} sweeps, shape {args.profile_shape}{cl}, "
          f"records every {jobs[0]['measure_every']} sweeps")


def headline(extras):
    """The side legs' figures in short, last on the JSON line."""
    h = {}
    b = extras.get("batched") or {}
    if "ratio" in b:
        h["batched_64_films"] = {"batched": round(b["batched"], 1), "plain": round(b["plain"], 1),
                                 "ratio": round(b["ratio"], 2), "alu_frac": round(b["batched_alu_frac"], 3)}
    s = extras.get("serving") or {}
    if "p50_latency_s" in s:
        h["serving_2000_jobs"] = {"attempts_per_ns": round(s["attempts_per_ns"], 1),
                                  "offered_attempts_per_ns": round(s["offered_attempts_per_ns"], 1),
                                  "p50_ms": round(1e3 * s["p50_latency_s"], 1),
                                  "p99_ms": round(1e3 * s["p99_latency_s"], 1)}
    c = extras.get("serving_capacity") or {}
    if "ratio" in c:
        h["served_vs_plain"] = {"served": round(c["served"], 1), "plain": round(c["plain"], 1),
                                "ratio": round(c["ratio"], 2)}
    p = extras.get("procedures") or {}
    for k in ("interface_tension_run", "contact_angle_run", "line_tension_run"):
        if k in p:
            h[k.replace("_run", "_set")] = {"attempts_per_ns": round(p[k]["attempts_per_ns"], 1),
                                           "alu_frac": round(p[k]["alu_frac"], 3)}
    t = extras.get("t_scan") or {}
    if "attempts_per_ns" in t:
        h["t_scan_40_films"] = {"attempts_per_ns": round(t["attempts_per_ns"], 1), "alu_frac": round(t["alu_frac"], 3)}
    o = extras.get("one_field_set") or {}
    if "autotuned" in o:
        h["contact_angle_one_field"] = {"autotuned": round(o["autotuned"], 1), "grid_best": round(o["grid_best"], 1),
                                        "ratio": round(o["ratio"], 2), "shape": o["shape"]}
    f = extras.get("film_8") or {}
    if "attempts_per_ns" in f:
        h["film_8"] = {"attempts_per_ns": round(f["attempts_per_ns"], 3)}
    h["unit"] = UNIT
    return h


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the batched/serving/e2e/cpu legs")
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--shape", default="auto", choices=["auto", "grid1", "grid2"],
                    help="launch shape of the 120x240x1600 film (auto: the library's autotuner); profiling "
                         "pins the autotuner's normal pick because ncu's serialisation distorts its timing")
    ap.add_argument("--profile-set", choices=PROFILE_SETS,
                    help="run one film set for ncu (see profile_set) instead of the benchmark")
    ap.add_argument("--profile-shape", default="grid2", choices=["grid1", "grid2", "gridq", "cluster"])
    ap.add_argument("--profile-cluster", type=int, default=0,
                    help="CTAs per film of --profile-shape cluster (0: the library's automatic size)")
    ap.add_argument("--profile-sweeps", type=int, default=4)
    ap.add_argument("--profile-every", type=int, default=None, help="record interval (0: no records)")
    ap.add_argument("--profile-lanes", type=int, default=1, help="batch lanes (0: the library's default)")
    args = ap.parse_args()
    if args.profile_set:
        profile_set(args)
        return
    if args.impl == "reference":
        reference_arm(args)
        return

    rank, world, local = dist_env()
    cpu = None
    if rank == 0 and not args.no_extras:
        cpu = cpu_baseline()  # before any GPU work in this process
    import torch
    import paper_1411_5588_gb300 as ig
    from paper_1411_5588_gb300 import workloads as WL

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    job = WL.film_46m(replica=rank)
    stream = torch.cuda.Stream()
    film = ig.Film(job["Lx"], job["Ly"], job["Lz"], job["J"], job["H1"], job["T"], job["seed"],
                   replica=job["replica"], stream=stream)
    film.init(job["init_kind"], job["flip_p"])
    # launch shapes picked by the library's autotuner (on a scratch film),
    # for the timed steps and for the update-kernel timing pass below
    if args.shape == "auto":
        code_step, code_kernel = film.autotune(SWEEPS_PER_STEP), film.autotune(0)
    else:
        code_step = code_kernel = {"grid1": ig.SHAPE_GRID_1, "grid2": ig.SHAPE_GRID_2}[args.shape]
        film.set_shape(code_step)
    shape_step, shape_kernel = SHAPE_NAMES[code_step], SHAPE_NAMES[code_kernel]
    sites = WL.sites(job)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            film.sweep(SWEEPS_PER_STEP, SWEEPS_PER_STEP)
        film.synchronize()
        film.read_series()
        film.reserve_records(args.steps)  # no series growth inside the timed steps
        events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
        sampler = ClockSampler(torch.cuda.current_device())
        sampler.start()
        time.sleep(0.4)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("bench_timed")  # ncu --nvtx-include bench_timed/ profiles these steps only
        for e0, e1 in events:
            flush.fill_(1)  # evict L2 (inputs smaller than L2)
            e0.record(stream)
            film.sweep(SWEEPS_PER_STEP, SWEEPS_PER_STEP)
            e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        if world > 1:
            torch.distributed.barrier()
        clocks = sampler.stop()
        step_ms = [e0.elapsed_time(e1) for e0, e1 in events]
        recs = film.read_series()
        assert recs.shape[0] == args.steps, recs.shape
        total_ms = max_over_ranks(sum(step_ms), device="cuda")
        value = world * sites * SWEEPS_PER_STEP * args.steps / (total_ms * 1e6)

        # update-kernel launch duration: sweeps without records are update
        # launches only (plus one counter-advance launch)
        n_k = 50
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        k0.record(stream)
        film.sweep(n_k, 0)
        k1.record(stream)
        torch.cuda.synchronize()
        upd_ms = k0.elapsed_time(k1) / (2 * n_k)
    ops_per_launch = OPS_PER_ATTEMPT * sites / 2
    achieved = ops_per_launch / (upd_ms * 1e-3) / 1e12
    peak = N_SM * LANES_PER_SM * SM_MAX_GHZ * 1e9 / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": profiled_traffic(code_kernel), "kernel": "update_film_kernel",
                "launch_us": upd_ms * 1e3, "ops_per_attempt": OPS_PER_ATTEMPT,
                "peak_from": "152 SMs x 128 int32 lanes x 2.07 GHz (nominal max clock)",
                "attempts_per_ns_at_peak": peak * 1e3 / OPS_PER_ATTEMPT}

    e2e = None
    extras = {}
    if not args.no_extras:
        # end to end through the C ABI on every rank: initial lattice from
        # pinned host memory, each step's record copied back to pinned host
        # memory on a copy stream, overlapping the next step's sweeps; the
        # time is the maximum over ranks
        host = torch.from_numpy(film.get_spins()).pin_memory()
        rl = 5 + job["Lx"]
        host_rec = torch.zeros((args.steps, rl), dtype=torch.int64).pin_memory()
        copy_stream = torch.cuda.Stream()
        film.reserve_records(args.steps)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        lib = ig.lib()
        ig.check(lib.ising_set_spins(film._h, ig.binding.P(host.data_ptr())), "ising_set_spins")
        got = 0
        for i in range(args.steps):
            film.sweep(SWEEPS_PER_STEP, SWEEPS_PER_STEP)
            got += film.read_series_async(host_rec[i].data_ptr(), 1, copy_stream)
        copy_stream.synchronize()
        film.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, device="cuda")
        assert got == args.steps and int(host_rec[-1, 0]) > 0
        e2e = {"value": world * sites * SWEEPS_PER_STEP * args.steps / dt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": world * sites / args.steps, "d2h_bytes_per_step": world * 8 * rl,
               "note": "initial int8 lattice uploaded once from pinned memory (bytes spread over the steps); "
                       "each step's record copied to pinned host memory (ising_read_series_async on a copy "
                       "stream, overlapping the next step); all ranks, time = max over ranks"}
    if rank == 0 and not args.no_extras:
        for name, fn in (("batched", lambda: batched_vs_plain(ig, WL, torch)),
                         ("serving", lambda: serving(ig, WL, n_jobs=args.serve_jobs)),
                         ("serving_capacity", lambda: serving_capacity(ig, WL)),
                         ("film_8", lambda: film_8_run(ig, WL)),
                         ("t_scan", lambda: t_scan_slice(ig, WL)),
                         ("procedures", lambda: procedures(ig, WL)),
                         ("one_field_set", lambda: one_field_set(ig, WL))):
            try:
                extras[name] = fn()
            except Exception as exc:  # report, never hide the main line
                extras[name] = {"error": repr(exc)}
    film.close()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    # per step: two half-sweep launches per sweep (the last one of the step
    # also takes the record sums), record_kernel, and the sweep-counter advance
    per_step_launches = 2 * SWEEPS_PER_STEP + 1 + 1
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "film 120x240x1600 (46,080,000 spins, bit-packed), Eq. 11 y boundary, "
                                   "free x with H1=+0.55/-0.55, periodic z, T=3, slab start + 1% flips, seed 2; "
                                   "step = 10 sweeps + one int64 record",
                       "sweeps_per_step": SWEEPS_PER_STEP, "l2": "flushed between steps (256 MiB write)",
                       "launch_shape": {"steps": shape_step, "kernel_timing": shape_kernel},
                       "parallelism": f"replicas x{world}"},
            "roofline": roofline, "clocks": clocks, "gpu_launches": per_step_launches * args.steps,
            "e2e": e2e, "cpu_baseline": cpu}
    line.update(extras)
    if extras:
        line["headline"] = headline(extras)  # last, so that a cut-off tail still shows it
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
