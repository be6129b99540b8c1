"""Writes the oracle's digests of the benchmark configurations' full runs.

TEST INFRASTRUCTURE.  Every value this script stores comes from the CPU
oracle (``oracle/``) alone; the seeded job lists come from the workload module
(``paper_1411_5588_gb300/workloads.py``, plain data, loaded here by path so
that the product package is never imported).  ``tests/test_gpu_full_runs.py``
runs the same chains through the C ABI and compares.

For each film it records the SHA-256 of
  - the record series: the (n_records, 5 + Lx) int64 array of the Eq. 1 /
    Eq. 17 sums (sweeps completed, B, M, M1, Mn, m(1..Lx)), little-endian,
    row-major;
  - the final spins: int8 in canonical order ((kx-1)*Ly + (ky-1))*Lz + (kz-1).
and, in plain numbers, the last record.

Usage (each configuration writes its own file ``digests_<name>.json``):
  python tests/golden/make_config_digests.py film_46m            # 2000 sweeps, a record every 10
  python tests/golden/make_config_digests.py ti_batch [sweeps]   # 64 films, 5000 sweeps, a record every sweep
  python tests/golden/make_config_digests.py t_scan_ends         # T = 1.5 and 4.4 films, 10^4 sweeps
  python tests/golden/make_config_digests.py contact_angle_one_field [sweeps]
                                          # the contact-angle set at H1 = 0.3: 10 films, 5000 sweeps
"""
from __future__ import annotations

import hashlib
import importlib.util
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def workloads():
    path = os.path.join(ROOT, "paper_1411_5588_gb300", "workloads.py")
    spec = importlib.util.spec_from_file_location("_seeded_workloads", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def sha256(a: np.ndarray, dtype) -> str:
    return hashlib.sha256(np.ascontiguousarray(a, dtype=np.dtype(dtype)).tobytes()).hexdigest()


def run_film(args):
    """One film through the oracle from its initial state; returns its entry."""
    index, job, n_sweeps, threads = args
    from oracle import oracle as O
    O.set_threads(threads)
    t0 = time.time()
    o = O.Film(job["Lx"], job["Ly"], job["Lz"], job["J"], job["H1"], job["T"], job["seed"], y_mode=job["y_mode"],
               replica=job["replica"])
    o.init(job["init_kind"], job["flip_p"])
    recs = o.sweep(n_sweeps, job["measure_every"])
    spins = o.get_spins()
    keys = ("Lx", "Ly", "Lz", "J", "H1", "T", "seed", "replica", "y_mode", "init_kind", "flip_p", "measure_every")
    return dict(index=index, job={k: job[k] for k in keys}, n_sweeps=int(n_sweeps), n_records=int(recs.shape[0]),
                records_sha256=sha256(recs, "<i8"), spins_sha256=sha256(spins, np.int8),
                last_record=[int(v) for v in recs[-1]] if recs.shape[0] else [],
                oracle_seconds=round(time.time() - t0, 1), oracle_threads=int(threads))


def main(argv):
    WL = workloads()
    name = argv[1]
    ncpu = os.cpu_count() or 1
    if name == "film_46m":
        job = WL.film_46m()
        todo = [(0, job, job["n_sweeps"], ncpu)]
        desc = "46M-site film 120x240x1600, T = 3, H1 = +0.55, slab start + 1% flips, seed 2, full run"
    elif name == "ti_batch":
        n = int(argv[2]) if len(argv) > 2 else 5000
        jobs = WL.ti_batch(n_sweeps=n)
        todo = [(i, j, n, 1) for i, j in enumerate(jobs)]
        desc = f"64-film integration set, every film, {n} sweeps with a record every sweep"
    elif name == "t_scan_ends":
        jobs = WL.t_scan_40()
        todo = [(i, jobs[i], jobs[i]["n_sweeps"], ncpu) for i in (0, len(jobs) - 1)]
        desc = "40-film temperature scan: the T = 1.5 and T = 4.4 films, full run (a record every sweep)"
    elif name == "contact_angle_one_field":
        n = int(argv[2]) if len(argv) > 2 else 5000
        jobs = WL.contact_angle_set(H1s=(0.3,), n_sweeps=n)["jobs"]
        todo = [(i, j, n, 1) for i, j in enumerate(jobs)]
        desc = f"contact-angle set at H1 = 0.3 (10 films 32x96x64), every film, {n} sweeps with a record every sweep"
    else:
        raise SystemExit(f"unknown configuration {name!r}")
    t0 = time.time()
    if len(todo) > 1 and todo[0][3] == 1:
        # independent films, one per process; spawn, so no worker inherits a
        # forked OpenMP runtime
        with mp.get_context("spawn").Pool(ncpu) as pool:
            entries = sorted(pool.map(run_film, todo, chunksize=1), key=lambda e: e["index"])
    else:
        entries = [run_film(a) for a in todo]
    with open(os.path.join(ROOT, "oracle", "ising_oracle.c"), "rb") as f:
        src_sha = hashlib.sha256(f.read()).hexdigest()
    out = dict(config=name, description=desc, written_by="tests/golden/make_config_digests.py (oracle only)",
               records_format="int64 little-endian, row-major (n_records, 5 + Lx): sweep, B, M, M1, Mn, m(1..Lx)",
               spins_format="int8, canonical order ((kx-1)*Ly + (ky-1))*Lz + (kz-1)",
               oracle_source_sha256=src_sha, wall_seconds=round(time.time() - t0, 1), cpus=ncpu, films=entries)
    path = os.path.join(HERE, f"digests_{name}.json")
    with open(path + ".tmp", "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    os.replace(path + ".tmp", path)
    print(path, out["wall_seconds"], "s")


if __name__ == "__main__":
    main(sys.argv)
