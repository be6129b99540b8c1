"""The seeded synthetic workloads match the recipes they state: the film
shapes, counts, parameter grids and distributions of the paper's runs
(Secs. II B-IV) that every parity test, procedure and benchmark draws from.
CPU only; nothing here runs the method."""
import numpy as np

from paper_1411_5588_gb300 import workloads as WL


def _valid(job):
    return job["Lx"] >= 1 and job["Ly"] >= 2 and job["Lz"] >= 2 and job["Lz"] % 2 == 0 and job["T"] > 0


def test_single_films():
    f8, f46 = WL.film_8(), WL.film_46m()
    assert WL.sites(f8) == 512 and f8["measure_every"] == 1 and f8["n_sweeps"] == 10000
    assert WL.sites(f46) == 46_080_000 and (f46["Lx"], f46["Ly"], f46["Lz"]) == (120, 240, 1600)
    assert f46["init_kind"] == WL.INIT_SLAB_Y and f46["flip_p"] == 0.01 and f46["measure_every"] == 10
    assert f46["y_mode"] == WL.Y_GAPBC and f46["H1"] == 0.55 and f46["T"] == 3.0
    assert WL.film_46m(replica=3)["replica"] == 3


def test_integration_set():
    jobs = WL.ti_batch()
    assert len(jobs) == 64 and all(_valid(j) for j in jobs)
    assert sorted({j["replica"] for j in jobs}) == list(range(64))
    for j in jobs:
        assert j["Lx"] in (32, 48, 64, 96) and j["Ly"] == 2 * j["Lx"] and j["Lz"] == 4 * j["Lx"]
    assert {j["T"] for j in jobs} == {2.0, 3.5} and {j["seed"] for j in jobs} == {1, 2}
    h = np.array(sorted({j["H1"] for j in jobs}))
    assert len(h) == 16 and 0 < h[0] and h[-1] < 0.75
    assert np.allclose(h + h[::-1], 0.75, atol=1e-14)  # Gauss-Legendre nodes are symmetric on [0, 0.75]
    t, _ = np.polynomial.legendre.leggauss(16)
    assert np.allclose(h, 0.375 * (np.sort(t) + 1.0), atol=1e-15)


def test_serving_stream():
    jobs = WL.serve_2000()
    assert len(jobs) == 2000 and all(_valid(j) for j in jobs)
    assert jobs == WL.serve_2000()  # seeded
    arr = np.array([j["arrival"] for j in jobs])
    assert arr[0] == 0.0 and np.all(np.diff(arr) >= 0)
    assert abs(np.diff(arr).mean() - 1 / 200) < 0.1 / 200  # Poisson at 200 jobs/s
    for key, lo, hi in (("Lx", 16, 96), ("Ly", 16, 192), ("Lz", 16, 768), ("n_sweeps", 500, 5000)):
        v = np.array([j[key] for j in jobs])
        assert v.min() >= lo and v.max() <= hi + (1 if key == "Lz" else 0), key
        # log-uniform: the median sits near the geometric mean of the range
        assert abs(np.log(np.median(v)) - 0.5 * np.log(lo * hi)) < 0.15, key
    T = np.array([j["T"] for j in jobs])
    H1 = np.array([j["H1"] for j in jobs])
    assert 1.5 <= T.min() and T.max() <= 4.2 and 0.0 <= H1.min() and H1.max() <= 1.0
    assert len({j["replica"] for j in jobs}) == 2000


def test_temperature_scan():
    jobs = WL.t_scan_40()
    T = np.array([j["T"] for j in jobs])
    assert len(jobs) == 40 and T[0] == 1.5 and abs(T[-1] - 4.4016) < 1e-12
    assert np.allclose(np.diff(T), 0.0744)
    assert all(WL.sites(j) == 46_080_000 for j in jobs)


def test_contact_angle_set():
    s = WL.contact_angle_set()
    jobs, roles = s["jobs"], s["roles"]
    assert len(jobs) == len(roles) == 40 and all(_valid(j) for j in jobs)
    assert all((j["Lx"], j["Ly"], j["Lz"], j["T"]) == (32, 96, 64, 3.0) for j in jobs)
    for j, h in enumerate(s["H1s"]):
        iface = jobs[roles.index(("interface", j))]
        plus = jobs[roles.index(("plus", j))]
        assert iface["y_mode"] == WL.Y_GAPBC and iface["init_kind"] == WL.INIT_SLAB_Y and iface["H1"] == h
        assert plus["y_mode"] == WL.Y_PBC and plus["init_kind"] == WL.INIT_ALL_UP and plus["H1"] == h
        nodes = [jobs[roles.index(("node", j, i))]["H1"] for i in range(s["n_gl"])]
        assert len(nodes) == 8 and all(0 < x < h for x in nodes)
        assert all(jobs[roles.index(("node", j, i))]["y_mode"] == WL.Y_PBC for i in range(s["n_gl"]))


def test_interface_tension_set():
    s = WL.interface_tension_set()
    jobs, roles = s["jobs"], s["roles"]
    assert len(jobs) == 192 and all(_valid(j) for j in jobs)
    betas = np.asarray(s["betas"])
    assert len(betas) == 24 and betas[0] == 0.2 and abs(betas[-1] - 1 / 3) < 1e-15
    for job, (name, si, k) in zip(jobs, roles):
        L = s["sizes"][si]
        assert (job["Lx"], job["Ly"], job["Lz"]) == (L, 60, L) and job["H1"] == 0.0
        assert abs(job["T"] - 1 / betas[k]) < 1e-12
        assert job["y_mode"] == {"apbc": WL.Y_APBC, "pbc": WL.Y_PBC}[name]


def test_line_tension_set():
    s = WL.line_tension_set()
    jobs, roles = s["jobs"], s["roles"]
    assert len(jobs) == 80 and all(_valid(j) for j in jobs)
    for Lx, Ly, Lz in s["sizes"]:
        assert Lx * Lz == 1536 and Ly * Lz == 9216  # the constant-area set
    for job, role in zip(jobs, roles):
        Lx, Ly, Lz = s["sizes"][role[1]]
        assert (job["Lx"], job["Ly"], job["Lz"]) == (Lx, Ly, Lz)
        assert 0 < job["H1"] < s["H1"]
        want = (WL.Y_GAPBC, WL.INIT_SLAB_Y) if role[0] == "interface" else (WL.Y_PBC, WL.INIT_ALL_UP)
        assert (job["y_mode"], job["init_kind"]) == want
