"""Run one film set as a batch for a few sweeps in a given launch shape: the
64-film integration set (16 H1 nodes x 2 T x 2 seeds, Lx 32..96) or one of
the procedure sets at the paper's sizes (contact angle, beta integration,
line tension), records after every sweep unless --every says otherwise
(0: none), in one lane unless --lanes says otherwise (so that one launch
covers the whole set).  The command the batch kernels' ncu summaries in
profiles/ were captured from.

    python -m paper_1411_5588_gb300.profile_batch [--set ti64] [--shape grid2] [--sweeps 4] [--every N] [--lanes L]
"""
from __future__ import annotations

import argparse

from . import binding as ig
from . import workloads as WL

SHAPES = {"grid1": ig.SHAPE_GRID_1, "grid2": ig.SHAPE_GRID_2, "gridq": ig.SHAPE_GRID_Q}
SETS = {
    "ti64": lambda n: WL.ti_batch(n_sweeps=n),
    "contact_angle": lambda n: WL.contact_angle_set(n_sweeps=n)["jobs"],
    "interface_tension": lambda n: WL.interface_tension_set(n_sweeps=n)["jobs"],
    "line_tension": lambda n: WL.line_tension_set(n_sweeps=n)["jobs"],
}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--set", default="ti64", choices=sorted(SETS))
    ap.add_argument("--shape", default="grid2", choices=sorted(SHAPES))
    ap.add_argument("--sweeps", type=int, default=4)
    ap.add_argument("--every", type=int, default=None, help="record interval (0: no records)")
    ap.add_argument("--lanes", type=int, default=1, help="batch lanes (0: the library's default)")
    args = ap.parse_args()
    jobs = SETS[args.set](args.sweeps)
    if args.every is not None:
        jobs = [dict(j, measure_every=args.every) for j in jobs]
    b = ig.Batch(jobs, lanes=args.lanes)
    b.set_shape(SHAPES[args.shape])
    if args.every != 0:
        b.reserve_records(args.sweeps)
    b.sweep(args.sweeps, False)
    b.synchronize()
    lanes = b.lanes
    b.close()
    print(f"{args.set}: {len(jobs)} films in {lanes} lane(s), {args.sweeps} sweeps, shape {args.shape}, "
          f"records every {jobs[0]['measure_every']} sweeps")


if __name__ == "__main__":
    main()
