"""Run the 64-film integration set (16 H1 nodes x 2 T x 2 seeds, Lx 32..96)
as one batch for a few sweeps in a given launch shape; the command the
multi-film update kernel's ncu summary in profiles/ was captured from.

    python -m paper_1411_5588_gb300.profile_batch [--shape grid2] [--sweeps 4]
"""
from __future__ import annotations

import argparse

from . import binding as ig
from . import workloads as WL

SHAPES = {"grid1": ig.SHAPE_GRID_1, "grid2": ig.SHAPE_GRID_2, "gridq": ig.SHAPE_GRID_Q}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", default="grid2", choices=sorted(SHAPES))
    ap.add_argument("--sweeps", type=int, default=4)
    args = ap.parse_args()
    jobs = WL.ti_batch(n_sweeps=args.sweeps)
    b = ig.Batch(jobs)
    b.set_shape(SHAPES[args.shape])
    b.sweep(args.sweeps, False)
    b.synchronize()
    b.close()
    print(f"{len(jobs)} films, {args.sweeps} sweeps, shape {args.shape}")


if __name__ == "__main__":
    main()
