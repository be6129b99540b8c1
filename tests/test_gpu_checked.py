"""The library built with ISING_CHECKED (every lattice word index of the
update, resident, cluster and record kernels and of the allocation-free
measurement tested against its plane): all parity
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
# the cluster-resident path: one CTA per film, then three (films of three
# layers or more), against the oracle
for C, sub in ((1, specs), (3, [f for f in specs if f["Lx"] >= 3])):
    sub = [dict(f, measure_every=1 + i % 2) for i, f in enumerate(sub)]
    b = ig.Batch(sub, lanes=1)
    b.set_cluster_size(C)
    b.set_shape(ig.SHAPE_CLUSTER)
    b.sweep(5, False)
    for i, f in enumerate(sub):
        o = R._oracle(f)
        assert np.array_equal(b.read_series(i), o.sweep(5, f["measure_every"])), (C, f)
        assert np.array_equal(b.get_spins(i), o.get_spins()), (C, f)
        films += 1
    b.close()
# the allocation-free measurement (its own kernel, the same record code)
import ctypes
import torch
for Lx, Ly, Lz, ym, xm in ((24, 32, 130, 0, 0), (12, 18, 70, 2, 1), (8, 256, 512, 1, 0), (7, 9, 2, 0, 0)):
    g = ig.Film(Lx, Ly, Lz, 1.0, 0.45, 2.8, 13, y_mode=ym, x_mode=xm)
    g.init(ig.INIT_SLAB_Y, 0.05)
    g.sweep(3, 0)
    packed = torch.empty(g.packed_words(), dtype=torch.int32, device="cuda")
    rec = torch.zeros(5 + Lx, dtype=torch.int64, device="cuda")
    g.get_packed_device(packed.data_ptr())
    g.synchronize()
    ig.check(ig.lib().ising_measure_packed_noalloc(ctypes.c_void_p(packed.data_ptr()), Lx, Ly, Lz, ym, xm,
                                                   g.sweep_count, ctypes.c_void_p(rec.data_ptr()), None),
             "ising_measure_packed_noalloc")
    torch.cuda.synchronize()
    assert np.array_equal(rec.cpu().numpy(), g.measure()), (Lx, Ly, Lz)
    g.close()
    films += 1
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


MAX_CHILD = r"""
import json, sys
sys.path.insert(0, __ROOT__)
import torch
import paper_1411_5588_gb300.binding as bd
bd.LIB_PATH = __LIB__
import paper_1411_5588_gb300 as ig
# 16384 x 32767 rows of 4 full words: 2^31 - 65536 words per parity plane,
# just under the largest film the library accepts (137e9 spins, 17 GB)
Lx, Ly, Lz = 16384, 32767, 256
film = ig.Film(Lx, Ly, Lz, 1.0, 0.4, float("inf"), 3)
film.init(ig.INIT_RANDOM)
n = film.packed_words()
before = torch.empty(n, dtype=torch.int32, device="cuda")
after = torch.empty_like(before)
film.get_packed_device(before.data_ptr())
r0 = film.measure()
film.sweep(1, 1)
film.get_packed_device(after.data_ptr())
r1 = film.read_series()[0]
film.synchronize()
flipped = True
step = 1 << 28
for i in range(0, n, step):
    flipped = flipped and bool(torch.equal(after[i:i + step], torch.bitwise_not(before[i:i + step])))
checked, count, first = ig.check_counters()
film.close()
print(json.dumps({"checked": checked, "count": count, "first": first, "words": n, "flipped": flipped,
                  "r0": [int(v) for v in r0[:8]], "r1": [int(v) for v in r1[:8]],
                  "m_negated": bool((r1[5:] == -r0[5:]).all())}))
"""


def test_largest_film_flips_every_site_at_infinite_temperature():
    """The largest class of film (just under 2^31 words per parity plane, where
    32-bit word indices are tightest), in the checked build: at beta = 0 every
    move is taken, so one sweep flips every site exactly once (each site sits
    in exactly one of the four phases).  The packed lattice must come out as
    its bitwise complement, the bond sum unchanged and every magnetisation sum
    negated, with not one out-of-range access."""
    from paper_1411_5588_gb300 import build
    lib = build.build(checked=True)
    code = MAX_CHILD.replace("__ROOT__", repr(ROOT)).replace("__LIB__", repr(lib))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["checked"] and out["count"] == 0, f"out-of-range lattice accesses: {out}"
    assert out["words"] == 2 * 16384 * 32767 * 4
    assert out["flipped"]
    r0, r1 = out["r0"], out["r1"]
    assert r0[0] == 0 and r1[0] == 1
    assert r1[1] == r0[1]  # B
    assert r1[2:5] == [-v for v in r0[2:5]]  # M, M1, Mn
    assert out["m_negated"]
    assert abs(r0[2]) < 16384 * 32767 * 256 // 100  # a random start
