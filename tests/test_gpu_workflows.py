"""The paper's procedures on the GPU path vs the oracle: every film's records
bit-identical, every FP64 result of the reduction within 1e-12 relative.
Small sets run their whole schedule; the default (benchmark-size) sets run
three sweeps of every film."""
import numpy as np
import pytest

from oracle import analysis as OA
from oracle import workflows as OW
from paper_1411_5588_gb300 import analysis as A
from paper_1411_5588_gb300 import workflows as PW
from paper_1411_5588_gb300 import workloads as WL

pytestmark = pytest.mark.gpu
REL = 1e-12


def agree(a, b):
    for k in b:
        x, y = np.asarray(a[k], dtype=np.float64), np.asarray(b[k], dtype=np.float64)
        assert x.shape == y.shape, k
        ok = np.isnan(y) & np.isnan(x) | (np.abs(x - y) <= REL * np.maximum(np.abs(y), 1.0))
        assert np.all(ok), (k, x, y)


def same_records(wl):
    g, o = PW.run(wl), OW.run(wl)
    for i, (a, b) in enumerate(zip(g, o)):
        assert np.array_equal(a, b), (wl["kind"], i, wl["roles"][i])
    return g, o


def test_contact_angle_procedure():
    wl = WL.contact_angle_set(Lx=6, Ly=16, Lz=8, H1s=(0.3, 0.6), n_gl=3, n_sweeps=300, first=100)
    g, o = same_records(wl)
    agree(PW.contact_angle(wl, g, 0.9), OW.contact_angle(wl, o, 0.9))


def test_interface_tension_procedure():
    wl = WL.interface_tension_set(sizes=(4, 6), Ly=8, n_beta=5, n_sweeps=300, first=100)
    g, o = same_records(wl)
    agree(PW.interface_tension(wl, g), OW.interface_tension(wl, o))


def test_line_tension_procedure():
    wl = WL.line_tension_set(sizes=((8, 32, 4), (4, 16, 8)), H1=0.45, n_gl=3, n_sweeps=300, first=100)
    g, o = same_records(wl)
    agree(PW.line_tension(wl, g, 1.2, 0.95, 0.9), OW.line_tension(wl, o, 1.2, 0.95, 0.9))


@pytest.mark.parametrize("make", [WL.contact_angle_set, WL.interface_tension_set, WL.line_tension_set])
def test_benchmark_size_sets_first_sweeps(make):
    wl = make(n_sweeps=3, first=0)
    same_records(wl)


def test_stiffness_steps_and_critical_field_from_gpu_records():
    """Secs. III B-C on the GPU path: the contact angles and gamma(theta) of a
    four-field scan, from GPU records, give the stiffness c and kappa
    (Eqs. 23-24), the step free energy and flat tension (Eq. 26), the step
    model's phi and H1* (Eqs. 28-32) and the critical field of the scan
    (Sec. III C, Eq. 32) within 1e-12 of the oracle's."""
    wl = WL.contact_angle_set(Lx=6, Ly=16, Lz=8, H1s=(0.2, 0.4, 0.6, 0.8), n_gl=3, n_sweeps=300, first=100)
    g, o = same_records(wl)
    gp, op = PW.contact_angle(wl, g, 0.9), OW.contact_angle(wl, o, 0.9)
    agree(gp, op)
    args = (wl["T"], wl["Lx"], wl["Lz"], wl["H1s"])
    agree(PW.stiffness_and_steps(gp["theta"], gp["gamma"], 0.9, *args),
          OW.stiffness_and_steps(op["theta"], op["gamma"], 0.9, *args))
    # a tolerance between the first point's tilt and the largest, half-way
    # between two neighbouring tilts so that rounding cannot move the crossing
    tilt = np.sort(np.pi / 2 - op["theta"])
    t0 = np.pi / 2 - op["theta"][0]
    above = tilt[tilt > t0]
    assert above.size, "no tilt beyond the first point's"
    tol = 0.5 * (t0 + above[0])
    H1 = np.asarray(wl["H1s"])
    agree(dict(zip("hf", A.critical_field(H1, gp["theta"], tol, wl["T"], wl["Lx"], wl["Lz"]))),
          dict(zip("hf", OA.critical_field(H1, op["theta"], tol, wl["T"], wl["Lx"], wl["Lz"]))))
