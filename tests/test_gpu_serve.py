"""Continuous batching: jobs that arrive while others run share the persistent
launch, and each job's result equals the result of running it alone."""
import numpy as np
import pytest

from paper_2505_05919_gb300 import Lattice
from paper_2505_05919_gb300.serve import Job, Server

pytestmark = pytest.mark.gpu


def _alone(job):
    with Lattice(job.cvf()) as lat:
        lat.sweep(job.sweeps)
        return lat.state(), lat.observables()


def _check_same(job):
    s, o = _alone(job)
    assert np.array_equal(job.state, s), job.id
    for k in ("sweep", "n_hb_raw", "n_coop", "acc_sigma", "acc_volume", "g", "n_state"):
        assert job.observables[k] == o[k], (job.id, k)
    for k in ("V_iso", "V", "U_LJ", "H"):
        assert abs(job.observables[k] - o[k]) <= 1e-12 * abs(o[k]), (job.id, k)


def _jobs(n, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        out.append(Job(T=float(rng.uniform(270, 330)), P=float(rng.uniform(0.1, 50)),
                       L=int(rng.choice([16, 32, 64, 96])), sweeps=int(rng.integers(20, 400)),
                       seed=7000 + i, keep_state=True))
    return out


def test_jobs_joining_midway_match_solo_runs():
    jobs = _jobs(10)
    srv = Server(epoch_steps=37)
    try:
        # three waves: later jobs join while earlier ones are part-way through
        for j in jobs[:4]:
            srv.submit(j)
        srv.step()
        srv.step()
        for j in jobs[4:8]:
            srv.submit(j)
        srv.step()
        for j in jobs[8:]:
            srv.submit(j)
        while srv.busy():
            srv.step()
    finally:
        srv.close()
    assert len(srv.finished) == len(jobs)
    # the mix really overlapped: some epoch advanced old and new jobs together
    assert max(j.admitted for j in jobs) < max(j.finished for j in jobs[:4])
    for j in jobs:
        _check_same(j)


def test_memory_budget_admission_and_cancel():
    jobs = _jobs(6, seed=3)
    per = max(j.device_bytes for j in jobs)
    srv = Server(epoch_steps=50, mem_budget_bytes=2 * per)  # at most two resident
    try:
        for j in jobs:
            srv.submit(j)
        srv.step()
        assert len(srv.resident) <= 2 and len(srv.waiting) >= 4
        victim = jobs[-1]
        assert srv.cancel(victim.id)
        while srv.busy():
            srv.step()
            assert srv.held_bytes <= 2 * per
    finally:
        srv.close()
    assert victim not in srv.finished and len(srv.finished) == len(jobs) - 1
    for j in srv.finished:
        _check_same(j)


def test_trace_summary():
    jobs = _jobs(8, seed=5)
    for i, j in enumerate(jobs):
        j.arrival = 0.002 * i
        j.keep_state = False
    srv = Server(epoch_steps=64)
    try:
        stats = srv.run_trace(jobs, time_limit=120)
    finally:
        srv.close()
    assert stats["jobs_finished"] == 8 and stats["jobs_waiting"] == 0
    assert stats["latency_p50_s"] > 0 and stats["latency_p99_s"] >= stats["latency_p50_s"]
    assert stats["replica_sweeps_per_s"] > 0
    assert stats["jobs_censored"] == 0 and not stats["latency_all_is_lower_bound"]
    assert stats["latency_all_p50_s"] == stats["latency_p50_s"]
    assert 0.0 < stats["gpu_busy_per_wall_s"] <= 1.05


def _obs_same(job):
    _, o = _alone(job)
    for k in ("sweep", "n_hb_raw", "n_coop", "acc_sigma", "acc_volume", "g", "n_state"):
        assert job.observables[k] == o[k], (job.id, k)
    for k in ("V_iso", "V", "U_LJ", "H"):
        assert abs(job.observables[k] - o[k]) <= 1e-12 * abs(o[k]), (job.id, k)


@pytest.mark.parametrize("overlap", [True, False])
def test_pipelined_epochs_match_solo_runs(overlap):
    """With overlap on, epoch k+1 is enqueued before epoch k's results are
    read; every job's observables (read back through tickets, no state
    copies) still equal its solo run, zero-step jobs included."""
    jobs = _jobs(12, seed=9)
    for j in jobs:
        j.keep_state = False
    jobs[5].sweeps = 0
    srv = Server(epoch_steps=29, overlap=overlap)
    try:
        for j in jobs[:5]:
            srv.submit(j)
        srv.step()
        for j in jobs[5:9]:
            srv.submit(j)
        srv.step()
        srv.step()
        for j in jobs[9:]:
            srv.submit(j)
        while srv.busy():
            srv.step()
    finally:
        srv.close()
    assert len(srv.finished) == len(jobs) and not srv.inflight
    assert srv.gpu_busy_s > 0
    for j in jobs:
        assert j.done == j.sweeps
        _obs_same(j)


def test_never_fitting_job_is_refused():
    jobs = _jobs(3, seed=11)
    big = Job(T=300.0, P=0.1, L=4096, sweeps=10, seed=1)
    srv = Server(epoch_steps=50, mem_budget_bytes=max(j.device_bytes for j in jobs))
    try:
        srv.submit(big)
        for j in jobs:
            srv.submit(j)
        assert big.error and big in srv.rejected and big not in srv.waiting
        while srv.busy():
            srv.step()
    finally:
        srv.close()
    assert len(srv.finished) == 3 and big.finished is None


def test_censored_latency_is_reported():
    """Under a time limit that ends the run early, the all-arrived latency
    percentiles count unfinished jobs with the time they waited (a lower
    bound), and say so."""
    jobs = [Job(T=300.0, P=0.1, L=1024, sweeps=50000, seed=100 + i, arrival=0.001 * i)
            for i in range(6)]
    jobs.append(Job(T=300.0, P=0.1, L=16, sweeps=10, seed=99, arrival=0.0))
    srv = Server(epoch_steps=100)
    try:
        stats = srv.run_trace(jobs, time_limit=0.5)
    finally:
        srv.close()
    assert stats["jobs_arrived"] == 7
    assert stats["jobs_censored"] >= 1 and stats["latency_all_is_lower_bound"]
    assert stats["jobs_finished"] + stats["jobs_censored"] == 7
    assert stats["latency_all_p99_s"] >= 0.45
    assert 0.0 < stats["gpu_busy_per_wall_s"] <= 1.05
