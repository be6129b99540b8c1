"""The library built with ISING_CHECKED (every lattice word index of the
update, resident and record kernels tested against its plane): all parity
shapes and a set of random films, every launch shape, bit-identical to the
oracle, and not one out-of-range access.  Runs in a child process, because a
process loads one build of the library."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
sys.path.insert(0, __ROOT__)
sys.path.insert(0, __ROOT__ + "/tests")
import numpy as np
import paper_1411_5588_gb300.binding as bd
bd.LIB_PATH = __LIB__
import paper_1411_5588_gb300 as ig
from oracle import oracle as O
import test_gpu_parity as P
import test_gpu_random as R
films = 0
for case in P.CASES:
    for shape in P.SHAPES:
        g, o = P._pair(case, shape=shape)
        for n, m in ((3, 1), (9, 2)):
            g.sweep(n, m)
            assert np.array_equal(g.read_series(), o.sweep(n, m)), (case, shape)
        assert np.array_equal(g.get_spins(), o.get_spins()), (case, shape)
        g.close()
        films += 1
specs = R._films(31, 16)
b = ig.Batch([dict(f, measure_every=i % 3) for i, f in enumerate(specs)])
for shape in (ig.SHAPE_GRID_1, ig.SHAPE_GRID_2, ig.SHAPE_GRID_Q):
    b.set_shape(shape)
    b.sweep(4, False)
b.close()
checked, count, first = ig.check_counters()
print(json.dumps({"checked": checked, "count": count, "first": first, "films": films}))
"""


def test_checked_build_has_no_out_of_range_access():
    from paper_1411_5588_gb300 import build
    lib = build.build(checked=True)
    code = CHILD.replace("__ROOT__", repr(ROOT)).replace("__LIB__", repr(lib))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["checked"] and out["films"] > 0
    assert out["count"] == 0, f"out-of-range lattice accesses: {out}"
