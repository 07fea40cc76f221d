"""Serving: concurrent jobs give the same result as the same job alone.

Jobs from two host threads run on a server with several slots (their kernels
overlap on the GPU); each result is compared with the job run alone through
a context of its own (and, for some, with the CPU oracle).  Merges sum with
FP64 atomics, so results agree to 1e-10 rather than bit for bit.
"""
import threading
import time

import numpy as np
import pytest

import oracle
import paper_2512_12094_gb300 as pp
import pp_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pp.build()
    pp.load()
    oracle.build()


def workload(kind, n, steps, eps, seed):
    rng = np.random.default_rng(seed)
    if kind == "ring":
        a = rng.uniform(0.1, 1.2, size=3)
        return pi.config1_ring(n=n, steps=steps, theta_j=a[0], theta_x=a[1], theta_z=a[2],
                               eps=eps, max_weight=8, symmetry=1)
    wl = pi.config0_heisenberg(n=n, dt=float(rng.uniform(0.02, 0.08)), steps=steps)
    wl.observable = pi.mean_z(n)
    wl.state = pi.neel_state(n)
    wl.eps = eps
    wl.symmetry = 2
    return wl


def job_of(wl, symmetry=None, mem_bytes=0):
    sym = wl.symmetry if symmetry is None else symmetry
    cfg = pp.pp_config_default(n_qubits=wl.circuit.n, symmetry=sym, coeff_eps=wl.eps,
                               max_weight=wl.max_weight)
    x, z, c = wl.observable.arrays()
    gx, gz, th = wl.circuit.gate_arrays(0)
    return pp.make_job(cfg, x, z, c, pp.pack_gates(gx, gz), th, len(wl.circuit.layers),
                       wl.state.bloch, True, mem_bytes)


def alone(wl, symmetry=None):
    sym = wl.symmetry if symmetry is None else symmetry
    p = pp.Propagator.from_workload(wl, symmetry=sym)
    v = p.run(wl)
    p.close()
    return v


def test_mixed_jobs_equal_alone():
    specs = [("ring", 12, 4, 1e-5, s) for s in range(6)] + \
            [("a2a", 8, 2, 0.0, s) for s in range(4)] + \
            [("ring", 32, 6, 1e-4, s) for s in range(4)] + \
            [("a2a", 10, 2, 1e-6, s) for s in range(2)]
    wls = [workload(*sp) for sp in specs]
    syms = [wl.symmetry if i % 3 else 0 for i, wl in enumerate(wls)]
    server = pp.pp_server_create(4, 4 << 30, 256 << 20)
    ids = [None] * len(wls)
    keep = []

    def submit(idx):
        for i in idx:
            job, bufs = job_of(wls[i], syms[i])
            keep.append(bufs)
            ids[i] = pp.pp_submit(server, job)

    threads = [threading.Thread(target=submit, args=(range(k, len(wls), 2),)) for k in range(2)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    results = [pp.pp_server_wait(server, jid) for jid in ids]
    pp.pp_server_destroy(server)
    for r, wl, sym in zip(results, wls, syms):
        assert r["done"] == 1 and r["status"] == 0
        assert r["value"] == pytest.approx(alone(wl, sym), abs=1e-10)
    # and against the oracle for the small ones
    for r, wl, sym in list(zip(results, wls, syms))[:6]:
        _, want = oracle.run_workload(wl, group=sym)
        assert r["value"] == pytest.approx(want, abs=1e-10)


def test_admission_limits_concurrency():
    wl = workload("ring", 16, 6, 1e-5, 1)
    server = pp.pp_server_create(4, 96 << 20, 0)  # room for one 64 MiB job at a time
    keep, ids = [], []
    for _ in range(4):
        job, bufs = job_of(wl, mem_bytes=64 << 20)
        keep.append(bufs)
        ids.append(pp.pp_submit(server, job))
    peak = 0
    for _ in range(2000):
        st = pp.pp_server_stats(server)
        peak = max(peak, st["running"])
        assert st["reserved_bytes"] <= 96 << 20
        if st["completed"] == 4:
            break
        time.sleep(0.001)
    res = [pp.pp_server_wait(server, j) for j in ids]
    pp.pp_server_destroy(server)
    assert peak <= 1
    assert len({r["value"] for r in res}) == 1 or \
        max(abs(r["value"] - res[0]["value"]) for r in res) < 1e-10


def test_oversized_job_is_rejected():
    server = pp.pp_server_create(2, 32 << 20, 0)
    job, bufs = job_of(workload("ring", 8, 1, 0.0, 0), mem_bytes=64 << 20)
    with pytest.raises(pp.PPError) as e:
        pp.pp_submit(server, job)
    assert e.value.status == 8  # PP_ERR_REJECTED
    pp.pp_server_destroy(server)


def test_reservation_grows_between_layers_without_restarting():
    """A job admitted with far too small a reservation finishes: its
    reservation is raised between layers (and a layer that runs out of room is
    applied again from the state before it), never from the first layer."""
    wl = workload("ring", 32, 10, 1e-4, 3)
    server = pp.pp_server_create(2, 2 << 30, 0)
    job, bufs = job_of(wl, mem_bytes=128 << 10)  # less than the job's tables will need
    r = pp.pp_server_wait(server, pp.pp_submit(server, job))
    pp.pp_server_destroy(server)
    assert r["status"] == 0, r["message"]
    assert r["reserved_bytes"] > 128 << 10
    assert r["grows"] >= 1 and r["restarts"] == 0
    assert r["value"] == pytest.approx(alone(wl), abs=1e-10)


def test_estimated_reservation_from_the_observable():
    """With no reservation named anywhere, a job is admitted with an estimate
    from its observable's size and grows from there."""
    wl = workload("ring", 24, 6, 1e-5, 4)
    server = pp.pp_server_create(2, 2 << 30, 0)
    job, bufs = job_of(wl)
    r = pp.pp_server_wait(server, pp.pp_submit(server, job))
    pp.pp_server_destroy(server)
    assert r["status"] == 0, r["message"]
    assert r["reserved_bytes"] >= 1 << 20 and r["restarts"] == 0
    assert r["value"] == pytest.approx(alone(wl), abs=1e-10)


def test_growing_job_is_not_starved_by_a_stream_of_small_jobs():
    """One job that must grow to most of the budget competes with small jobs
    that keep arriving: running jobs that wait for memory are served before
    new admissions, so it finishes; every result equals the job alone and the
    reservations never exceed the budget."""
    big = workload("ring", 32, 8, 1e-5, 5)
    p = pp.Propagator.from_workload(big, symmetry=1)
    want_big = p.run(big)
    big_bytes = p.stats()["device_bytes"]
    p.close()
    budget = int(2.5 * big_bytes) + (64 << 20)
    small = [workload("ring", 12, 3, 1e-5, 100 + k) for k in range(40)]
    server = pp.pp_server_create(4, budget, 0)
    keep = []
    job, bufs = job_of(big, mem_bytes=1 << 20)
    keep.append(bufs)
    big_id = pp.pp_submit(server, job)
    ids = []
    stop = threading.Event()
    peak = [0]

    def watch():
        while not stop.is_set():
            st = pp.pp_server_stats(server)
            peak[0] = max(peak[0], st["reserved_bytes"])
            time.sleep(0.0005)

    w = threading.Thread(target=watch)
    w.start()
    for wl in small:
        job, bufs = job_of(wl)
        keep.append(bufs)
        ids.append(pp.pp_submit(server, job))
        time.sleep(0.002)
    rb = pp.pp_server_wait(server, big_id)
    rs = [pp.pp_server_wait(server, j) for j in ids]
    stop.set()
    w.join()
    pp.pp_server_destroy(server)
    assert rb["status"] == 0, rb["message"]
    assert rb["grows"] >= 1
    assert rb["value"] == pytest.approx(want_big, abs=1e-10)
    assert peak[0] <= budget
    for r, wl in zip(rs, small):
        assert r["status"] == 0, r["message"]
        assert r["value"] == pytest.approx(alone(wl), abs=1e-10)


def test_short_job_is_admitted_before_a_long_one_submitted_earlier():
    """Admission follows the predicted run time: on a one-slot server busy
    with a first job, an expensive job (12 steps at n = 32, eps 1e-5) and then
    a cheap one (3 steps at n = 12, eps 1e-3) are queued; the cheap one starts
    first although it arrived later, and both results equal the jobs alone."""
    first = workload("ring", 16, 8, 1e-4, 7)
    slow = workload("ring", 32, 12, 1e-5, 8)
    fast = workload("ring", 12, 3, 1e-3, 9)
    server = pp.pp_server_create(1, 8 << 30, 0)
    keep, ids = [], []
    for wl in (first, slow, fast):
        job, bufs = job_of(wl)
        keep.append(bufs)
        ids.append(pp.pp_submit(server, job))
    res = [pp.pp_server_wait(server, j) for j in ids]
    pp.pp_server_destroy(server)
    for r in res:
        assert r["status"] == 0, r["message"]
    assert res[2]["queue_ms"] < res[1]["queue_ms"]
    for r, wl in zip(res, (first, slow, fast)):
        assert r["value"] == pytest.approx(alone(wl), abs=1e-10)
