"""The procedures' reductions on the host: the product's workflow code
(library calls) fed the oracle's records agrees with the oracle's own
workflow to 1e-12 relative.  The GPU runs of the same sets are in
test_gpu_workflows.py."""
import numpy as np
import pytest

from oracle import workflows as OW
from paper_1411_5588_gb300 import workflows as PW
from paper_1411_5588_gb300 import workloads as WL

REL = 1e-12


def small_sets():
    return (WL.contact_angle_set(Lx=6, Ly=16, Lz=8, H1s=(0.3, 0.6), n_gl=3, n_sweeps=300, first=100),
            WL.interface_tension_set(sizes=(4, 6), Ly=8, n_beta=5, n_sweeps=300, first=100),
            WL.line_tension_set(sizes=((8, 32, 4), (4, 16, 8)), H1=0.45, n_gl=3, n_sweeps=300, first=100))


def agree(a, b):
    for k in b:
        x, y = np.asarray(a[k], dtype=np.float64), np.asarray(b[k], dtype=np.float64)
        assert x.shape == y.shape, k
        ok = np.isnan(y) & np.isnan(x) | (np.abs(x - y) <= REL * np.maximum(np.abs(y), 1.0))
        assert np.all(ok), (k, x, y)


@pytest.fixture(scope="module")
def oracle_runs():
    sets = small_sets()
    return sets, [OW.run(wl) for wl in sets]


def test_contact_angle_reduction(oracle_runs):
    (ca, _, _), (rec, _, _) = oracle_runs
    agree(PW.contact_angle(ca, rec, 0.9), OW.contact_angle(ca, rec, 0.9))


def test_interface_tension_reduction(oracle_runs):
    (_, it, _), (_, rec, _) = oracle_runs
    agree(PW.interface_tension(it, rec), OW.interface_tension(it, rec))


def test_line_tension_reduction(oracle_runs):
    (_, _, lt), (_, _, rec) = oracle_runs
    agree(PW.line_tension(lt, rec, 1.2, 0.95, 0.9), OW.line_tension(lt, rec, 1.2, 0.95, 0.9))


def test_stiffness_and_steps_reduction():
    th = np.array([1.5, 1.4, 1.3, 1.2])
    g = 0.9 * (1 + 0.3 * (np.pi / 2 - th) ** 2)
    agree(PW.stiffness_and_steps(th, g, 0.9, 3.0, 32, 64, (0.1, 0.3)),
          OW.stiffness_and_steps(th, g, 0.9, 3.0, 32, 64, (0.1, 0.3)))


def test_sets_are_well_formed():
    for wl in small_sets() + (WL.contact_angle_set(), WL.interface_tension_set(), WL.line_tension_set()):
        assert len(wl["jobs"]) == len(wl["roles"]) == len(set(wl["roles"]))
        assert [j["replica"] for j in wl["jobs"]] == list(range(len(wl["jobs"])))
        assert all(j["Lz"] % 2 == 0 and j["T"] > 0 for j in wl["jobs"])
    lt = WL.line_tension_set()
    assert len({Lx * Lz for Lx, _, Lz in lt["sizes"]}) == 1 and len({Ly * Lz for _, Ly, Lz in lt["sizes"]}) == 1
