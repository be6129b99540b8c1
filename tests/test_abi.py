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
