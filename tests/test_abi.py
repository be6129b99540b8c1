"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/ising.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(ising_[a-z0-9_]+)\s*\(", text))
    return names


def test_build_and_exports():
    from paper_1411_5588_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    decl = _declared()
    assert len(decl) >= 40
    missing = [n for n in sorted(decl) if not hasattr(lib, n)]
    assert not missing, missing


def test_ptxas_report_has_no_spills():
    """Every kernel of the library fits its registers (no local-memory spills)."""
    from paper_1411_5588_gb300 import build
    build.build()
    rep = open(os.path.join(build.BUILD, "ising_kernels.o.ptxas.txt")).read()
    assert "sm_103a" in rep
    for m in re.finditer(r"(\d+) bytes spill stores, (\d+) bytes spill loads", rep):
        assert m.group(1) == "0" and m.group(2) == "0"


def test_strerror_and_version():
    import paper_1411_5588_gb300 as ig
    L = ig.lib()
    assert L.ising_strerror(ig.EINVAL) == b"invalid argument"
    ma, mi, sm = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    assert L.ising_version(ctypes.byref(ma), ctypes.byref(mi), ctypes.byref(sm)) == 0
    assert sm.value == 103


def _has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.mark.skipif(_has_gpu(), reason="checks behaviour without a device")
def test_create_without_device_reports_cuda_error():
    import paper_1411_5588_gb300 as ig
    with pytest.raises(ig.IsingError) as e:
        ig.Film(4, 4, 4, 1.0, 0.0, 3.0, 1)
    assert e.value.status == ig.ECUDA


def test_invalid_sizes_are_rejected_before_any_device_call():
    import paper_1411_5588_gb300 as ig
    for args in [(0, 4, 4), (4, 1, 4), (4, 4, 3), (4, 4, 0)]:
        with pytest.raises(ig.IsingError) as e:
            ig.Film(*args, 1.0, 0.0, 3.0, 1)
        assert e.value.status == ig.EINVAL
    with pytest.raises(ig.IsingError) as e:
        ig.Film(4, 4, 4, 1.0, 0.0, -1.0, 1)
    assert e.value.status == ig.EINVAL


def test_batch_lanes_above_the_limit_are_einval():
    """Checked before any device work, so it runs without a GPU."""
    import paper_1411_5588_gb300 as ig
    spec = dict(Lx=4, Ly=4, Lz=8, T=3.0, H1=0.1, seed=1, replica=0)
    with pytest.raises(ig.IsingError) as e:
        ig.Batch([spec], lanes=ig.MAX_LANES + 1)
    assert e.value.status == ig.EINVAL


@pytest.mark.skipif(_has_gpu(), reason="checks behaviour without a device")
def test_film_size_limit_is_exact():
    """At most 2^31 words per parity plane: 16384 x 32768 rows of four words
    reach it and are refused before any device call (EINVAL); one row fewer
    passes the check and only then meets the missing device (ECUDA)."""
    import paper_1411_5588_gb300 as ig
    with pytest.raises(ig.IsingError) as e:
        ig.Film(16384, 32768, 256, 1.0, 0.0, 3.0, 1)
    assert e.value.status == ig.EINVAL
    with pytest.raises(ig.IsingError) as e:
        ig.Film(16384, 32767, 256, 1.0, 0.0, 3.0, 1)
    assert e.value.status == ig.ECUDA


def test_batch_jobs_are_checked_before_any_device_call():
    """Every job of a batch is validated before the first device call, so a
    bad one is EINVAL even without a GPU (and with one, nothing is
    allocated)."""
    import paper_1411_5588_gb300 as ig
    good = dict(Lx=4, Ly=4, Lz=8, T=3.0, H1=0.1, seed=1, replica=0)
    bad = [dict(good, Lz=7), dict(good, Ly=1), dict(good, T=0.0), dict(good, y_mode=3),
           dict(good, x_mode=ig.X_PBC, Lx=3), dict(good, init_kind=5),
           dict(good, init_kind=ig.INIT_SLAB_Y, flip_p=1.5),
           dict(good, init_kind=ig.INIT_SLAB_Y, flip_p=float("nan")),
           dict(good, Lx=16384, Ly=32768, Lz=256)]
    for spec in bad:
        with pytest.raises(ig.IsingError) as e:
            ig.Batch([good, spec])
        assert e.value.status == ig.EINVAL, spec
    with pytest.raises(ig.IsingError) as e:
        ig.Batch([])
    assert e.value.status == ig.EINVAL


def test_cluster_size_calls_reject_null_handles():
    """The cluster-shape calls check their arguments before touching a batch
    (no device needed)."""
    import paper_1411_5588_gb300 as ig
    L = ig.lib()
    v = ctypes.c_uint32(7)
    assert L.ising_batch_set_cluster_size(None, 2) == ig.EINVAL
    assert L.ising_batch_get_cluster_size(None, ctypes.byref(v)) == ig.EINVAL
    assert v.value == 7
    assert ig.SHAPE_CLUSTER == 5
