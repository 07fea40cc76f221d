"""The job server's host-side rules on the CPU (no GPU).

paper_2512_12094_gb300/csrc/pp_admission.h holds the rules the server in
pp_server.cu applies: the cost model that predicts a queued job's run time,
the admission key with its credit for waiting, the choice of the job to admit
with the bypass limit, and the share of the GPU a layer takes.  The same
header is compiled here into a small driver (tests/admission_main.cpp) and
checked against a numpy solve of the ridge problem and against the rules'
stated properties.
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
PRIOR = np.array([-7.845, 0.887, 1.444, 0.703, 0.519, -0.438, -1.080, -0.338])
MAX_BYPASS = 8


@pytest.fixture(scope="module", params=["plain", "asan_ubsan"])
def driver(request, tmp_path_factory):
    """The driver built plainly, and with AddressSanitizer and
    UndefinedBehaviorSanitizer (no recovery: an invalid access or undefined
    behaviour ends the run with an error)."""
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    flags = ["-O1", "-std=c++17", "-Wall", "-Wextra", "-Werror"]
    if request.param == "asan_ubsan":
        flags += ["-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                  "-fno-omit-frame-pointer"]
    exe = str(tmp_path_factory.mktemp("admission_" + request.param) / "admission")
    r = subprocess.run(["g++", *flags, os.path.join(HERE, "admission_main.cpp"), "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0 and request.param == "asan_ubsan":
        pytest.skip("g++ without sanitizer runtimes: " + r.stderr.strip()[-200:])
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1")

    def run(text):
        out = subprocess.run([exe], input=text, capture_output=True, text=True, timeout=120,
                             env=env)
        assert out.returncode == 0, out.stderr
        assert "runtime error" not in out.stderr and "AddressSanitizer" not in out.stderr
        return [[float(v) for v in line.split()] for line in out.stdout.strip().splitlines()]
    return run


def _fit_request(F, y):
    rows = "\n".join(" ".join(repr(float(v)) for v in list(f) + [t]) for f, t in zip(F, y))
    return f"fit {len(y)}\n{rows}\n"


def test_cost_model_without_data_is_the_prior(driver):
    assert driver("fit 0\n")[0] == pytest.approx(PRIOR.tolist(), abs=0)


@pytest.mark.parametrize("n_obs,seed", [(1, 0), (5, 1), (40, 2), (400, 3)])
def test_cost_model_is_the_ridge_solution(driver, n_obs, seed):
    """After any number of finished jobs the coefficients minimise
    |F beta - y|^2 + |beta - prior|^2: (F^T F + I) beta = F^T y + prior."""
    rng = np.random.default_rng(seed)
    F = np.column_stack([np.ones(n_obs), rng.uniform(0, 4, n_obs), rng.uniform(2, 9, n_obs),
                         rng.uniform(5, 15, n_obs), rng.integers(0, 2, n_obs),
                         np.zeros(n_obs), rng.uniform(2, 5, n_obs), rng.integers(0, 2, n_obs)])
    F[:, 5] = F[:, 4] * F[:, 3]
    y = F @ rng.normal(size=8) + rng.normal(scale=0.3, size=n_obs)
    got = np.array(driver(_fit_request(F, y))[0])
    want = np.linalg.solve(F.T @ F + np.eye(8), F.T @ y + PRIOR)
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=1e-9)


def test_cost_model_learns_an_exact_law(driver):
    """Many jobs whose log run time follows a fixed linear law: the predicted
    log run times approach the law's.  (The prior still pulls, and correlated
    features share the intercept, so single coefficients move more than the
    predictions do.)"""
    rng = np.random.default_rng(7)
    n = 2000
    F = np.column_stack([np.ones(n), rng.uniform(0, 4, n), rng.uniform(2, 9, n),
                         rng.uniform(5, 15, n), rng.integers(0, 2, n), np.zeros(n),
                         rng.uniform(2, 5, n), rng.integers(0, 2, n)])
    F[:, 5] = F[:, 4] * F[:, 3]
    law = np.array([-3.0, 1.0, 1.0, 0.5, 2.0, -0.1, 0.25, -0.5])
    got = np.array(driver(_fit_request(F, F @ law))[0])
    rms = lambda e: float(np.sqrt(np.mean(e ** 2)))  # noqa: E731
    err, prior_err = F @ got - F @ law, F @ PRIOR - F @ law
    # within 3 % of the law's run times, and at least 20 times closer than the prior
    assert rms(err) < 0.03 and rms(err) < rms(prior_err) / 20


def test_features(driver):
    # ring n=32 job: 20 layers of 96 gates, eps 1e-4, no noise, Z_n
    got = driver("features 32 1 0 1e-4 20 96\n")[0]
    want = [1.0, math.log(20), math.log(96), math.log(1e4), 0.0, 0.0, math.log(32), 1.0]
    assert got == pytest.approx(want, rel=1e-14)
    # all-to-all n=64 with per-gate noise, eps 0 (counts as 1e-12), no group
    got = driver("features 64 0 1 0 10 6048\n")[0]
    le = math.log(1e12)
    want = [1.0, math.log(10), math.log(6048), le, 1.0, le, math.log(64), 0.0]
    assert got == pytest.approx(want, rel=1e-14)


def test_admission_key_ages_and_puts_returned_jobs_first(driver):
    out = driver("key 2.5 0 0\nkey 2.5 10 0\nkey 2.5 35 0\nkey 9.0 0 1\n")
    assert [o[0] for o in out[:3]] == pytest.approx([2.5, 1.5, 2.5 - 3.5])
    assert out[3][0] < -1e8


def _pick(driver, jobs):
    text = f"pick {len(jobs)}\n" + "".join(f"{k!r} {int(f)} {b}\n" for k, f, b in jobs)
    out = driver(text)[0]
    return int(out[0]), [int(v) for v in out[1:]]


def test_pick_takes_the_lowest_key_that_fits(driver):
    jobs = [(3.0, True, 0), (1.0, False, 0), (2.0, True, 0), (0.5, False, 2)]
    pick, byp = _pick(driver, jobs)
    # order by key: job 3 (no room), job 1 (no room), job 2 (fits)
    assert pick == 2
    assert byp == [0, 1, 0, 3]


def test_pick_stops_behind_a_job_passed_too_often(driver):
    jobs = [(1.0, False, MAX_BYPASS), (2.0, True, 0)]
    pick, byp = _pick(driver, jobs)
    assert pick == -1 and byp == [MAX_BYPASS, 0]
    jobs = [(1.0, False, MAX_BYPASS - 1), (2.0, True, 0)]
    pick, byp = _pick(driver, jobs)
    assert pick == 1 and byp == [MAX_BYPASS, 0]


def test_pick_with_nothing_that_fits_or_an_empty_queue(driver):
    assert _pick(driver, [(1.0, False, 0), (2.0, False, 0)]) == (-1, [0, 0])
    assert driver("pick 0\n")[0] == [-1.0]


def test_pick_random_queues_follow_the_rule(driver):
    """On random queues the admitted job fits; every job before it in key
    order does not fit, is below the bypass limit and counts one bypass more;
    with no job admitted, the walk in key order met a job at the limit or no
    job fits."""
    rng = np.random.default_rng(11)
    for _ in range(200):
        q = int(rng.integers(1, 12))
        jobs = [(float(rng.normal()), bool(rng.random() < 0.4), int(rng.integers(0, MAX_BYPASS + 2)))
                for _ in range(q)]
        pick, byp = _pick(driver, jobs)
        order = sorted(range(q), key=lambda k: (jobs[k][0], k))
        if pick >= 0:
            assert jobs[pick][1]
            before = order[:order.index(pick)]
            for k in before:
                assert not jobs[k][1] and jobs[k][2] < MAX_BYPASS
            for k in range(q):
                assert byp[k] == jobs[k][2] + (1 if k in before else 0)
        else:
            assert byp == [j[2] for j in jobs]
            first_fit = next((r for r, k in enumerate(order) if jobs[k][1]), None)
            blocked = any(jobs[k][2] >= MAX_BYPASS for k in order[:first_fit])
            assert first_fit is None or blocked


@pytest.mark.parametrize("slots,running,wanted,free,want", [
    (8, 1, 1.0, 1024, 1024),   # alone: the whole GPU
    (8, 2, 1.0, 1024, 512),    # an equal share among the running jobs
    (8, 8, 1.0, 1024, 128),    # never below 1/slots
    (8, 2, 0.05, 1024, 128),   # a small launch still gets 1/slots
    (8, 2, 0.3, 1024, 308),    # no more than the launch would use
    (8, 2, 1.0, 300, 300),     # what is free when that is at least 1/slots
    (8, 2, 1.0, 127, 0),       # less than 1/slots free: wait
    (1, 1, 1.0, 1024, 1024),
    (1, 3, 0.1, 1023, 0),      # one slot: its share is the whole GPU
])
def test_share_units(driver, slots, running, wanted, free, want):
    assert driver(f"share {slots} {running} {wanted!r} {free}\n")[0][0] == want
