"""The serving loop's host logic on the CPU: admission in arrival order under
a memory budget, refusal of jobs that could never fit, epochs that split
long jobs, one epoch kept in flight with overlap on, cancellation,
zero-step jobs and the latency summary with censored jobs.  The GPU parts
(the batch of replicas, CUDA events and streams, the free-memory query) are
replaced by fakes that record what the server asks of them; the replicas'
arithmetic is covered by tests/test_gpu_serve.py."""
import numpy as np
import pytest
import torch

from paper_2505_05919_gb300 import serve
from paper_2505_05919_gb300.serve import Job, Server


class FakeEvent:
    clock = [0.0]

    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        FakeEvent.clock[0] += 1.0
        self.t = FakeEvent.clock[0]

    def elapsed_time(self, other):
        return other.t - self.t  # ms


class FakeStream:
    pass


class FakeBatch:
    """Replicas by slot; sweep() advances them at once, so a ticket taken
    right after an epoch sees that epoch's steps (as the stream order would)."""
    instances = []

    def __init__(self, params_list=(), stream=None):
        self.reps = {}
        self.n_slots = 0
        self.tickets = {}
        self.n_tickets = 0
        self.plans = []
        self.added = []
        self.tiles = None
        FakeBatch.instances.append(self)

    def set_tiles(self, c):
        self.tiles = c

    def add(self, p):
        rid = next(i for i in range(self.n_slots + 1) if i not in self.reps)
        self.n_slots = max(self.n_slots, rid + 1)
        self.reps[rid] = {"L": p.L, "steps": 0}
        self.added.append((rid, p.L))
        return rid

    def remove(self, rid):
        del self.reps[rid]

    def pool_bytes(self):
        return (0, 0)

    def slots(self):
        return self.n_slots

    def sweep(self, plan):
        assert len(plan) == self.n_slots
        for rid, n in enumerate(plan):
            if n:
                self.reps[rid]["steps"] += n
        self.plans.append(list(plan))

    def observables_enqueue(self, rids):
        self.n_tickets += 1
        t = self.n_tickets
        self.tickets[t] = [{"sweep": self.reps[r]["steps"], "L": self.reps[r]["L"]} for r in rids]
        return t

    def observables_collect(self, ticket, n):
        out = self.tickets.pop(ticket)
        assert len(out) == n
        return out

    def state(self, rid):
        L = self.reps[rid]["L"]
        return np.zeros((L, L), np.uint16)

    def close(self):
        pass


FREE = 64 << 30


@pytest.fixture
def fakes(monkeypatch):
    FakeBatch.instances.clear()
    monkeypatch.setattr(serve, "Batch", FakeBatch)
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a: (FREE, 2 * FREE))
    return FakeBatch


def job(L=64, sweeps=100, **kw):
    return Job(T=300.0, P=0.1, L=L, sweeps=sweeps, seed=1, **kw)


def run_until_idle(srv, limit=1000):
    for _ in range(limit):
        if not srv.busy():
            break
        srv.step()
    srv.drain()


def test_admission_in_arrival_order_under_a_budget(fakes):
    one = job(L=64).device_bytes
    srv = Server(epoch_steps=50, mem_budget_bytes=2 * one + 10)
    jobs = [job(L=64, sweeps=100 + i) for i in range(5)]
    for j in jobs:
        srv.submit(j)
    srv.step()
    assert len(srv.resident) == 2 and [j.id for j in srv.resident.values()] == [0, 1]
    run_until_idle(srv)
    assert [j.id for j in srv.finished] == [0, 1, 2, 3, 4]
    for j in jobs:
        assert j.observables["sweep"] == j.sweeps and j.done == j.sweeps
    assert srv.held_bytes == 0 and srv.resident_cells == 0 and not srv.resident
    assert max(srv.queue_len) == 3


def test_a_job_that_can_never_fit_is_refused_not_queued(fakes):
    small = job(L=64)
    srv = Server(mem_budget_bytes=small.device_bytes * 4)
    big = job(L=4096)
    srv.submit(big)
    srv.submit(small)
    assert big.error and big in srv.rejected and big not in srv.waiting
    assert srv.submit(job(L=64, sweeps=-1)) >= 0 and srv.rejected[-1].error
    run_until_idle(srv)
    assert small.finished is not None and small.observables["sweep"] == small.sweeps
    s = srv.summary()
    assert s["jobs_rejected"] == 2 and s["jobs_finished"] == 1


def test_epochs_split_long_jobs_and_run_new_ones_alongside(fakes):
    srv = Server(epoch_steps=200)
    a = job(sweeps=450)
    srv.submit(a)
    srv.step()                  # epoch 1: a 200
    b = job(sweeps=150)
    srv.submit(b)
    srv.step()                  # epoch 2: a 200, b 150 (b joins half-way through a)
    run_until_idle(srv)         # epoch 3: a 50
    batch = fakes.instances[-1]
    ra, rb = batch.added[0][0], batch.added[1][0]
    assert [p[ra] for p in batch.plans] == [200, 200, 50]
    assert [p[rb] for p in batch.plans if len(p) > rb] == [150, 0]
    assert a.observables["sweep"] == 450 and b.observables["sweep"] == 150
    assert b.finished <= a.finished


def test_overlap_keeps_one_epoch_in_flight(fakes):
    srv = Server(epoch_steps=10)
    srv.submit(job(sweeps=100))
    srv.step()
    assert len(srv.inflight) == 1          # enqueued, not waited for
    srv.step()
    assert len(srv.inflight) == 1          # the previous one retired
    off = Server(epoch_steps=10, overlap=False)
    off.submit(job(sweeps=100))
    off.step()
    assert len(off.inflight) == 0          # waits for the epoch it enqueued


def test_epoch_length_follows_the_resident_cells(fakes):
    srv = Server(epoch_steps=1000, epoch_cell_steps=64 * 64 * 30)
    srv.submit(job(L=64, sweeps=100))
    srv.submit(job(L=64, sweeps=100))
    srv.step()
    batch = fakes.instances[-1]
    assert max(batch.plans[0]) == 15      # 30 steps' worth of one lattice, shared by two


def test_cancel_waiting_and_resident_jobs(fakes):
    one = job(L=64).device_bytes
    srv = Server(epoch_steps=10, mem_budget_bytes=one + 10)
    a, b = job(sweeps=100), job(sweeps=100)
    srv.submit(a)
    srv.submit(b)
    srv.step()                             # a resident, b waiting
    assert srv.cancel(b.id) and b.cancelled and b not in srv.waiting
    assert srv.cancel(a.id) and a.cancelled and not srv.resident
    assert not srv.cancel(12345)
    run_until_idle(srv)
    assert a.finished is None and b.finished is None and not srv.finished
    assert srv.summary()["jobs_censored"] == 0   # cancelled jobs are not waiting for service


def test_zero_step_jobs_finish_with_their_initial_state(fakes):
    srv = Server(epoch_steps=10)
    z = job(sweeps=0, keep_state=True)
    srv.submit(z)
    run_until_idle(srv)
    assert z.finished is not None and z.observables["sweep"] == 0
    assert z.state is not None and z.state.shape == (64, 64)
    assert not any(any(p) for p in fakes.instances[-1].plans)


def test_latency_over_all_arrivals_is_a_lower_bound_with_censored_jobs(fakes):
    srv = Server(epoch_steps=10)
    done = job(sweeps=10, arrival=0.0)
    left = job(sweeps=10 ** 6, arrival=0.0)
    srv.arrived = [done, left]
    srv.submit(done)
    srv.submit(left)
    for _ in range(3):
        srv.step()
    srv.drain()
    s = srv.summary()
    assert s["jobs_finished"] == 1 and s["jobs_censored"] == 1
    assert s["latency_all_is_lower_bound"]
    assert s["latency_p50_s"] == pytest.approx(done.latency)
    assert s["latency_all_p99_s"] >= s["latency_p99_s"]
