"""Continuous-batching request loop for equation-of-state scan jobs.

Jobs (a state point (T, P), a lattice side L, a number of MC steps, a seed)
arrive over time.  The server keeps every admitted job's lattice resident on
the device as one replica of a Batch.  Each call of step()

  1. admits waiting jobs in arrival order while free HBM (minus a reserve)
     covers the new replica and a slot is free; the replica's allocation and
     initialisation are enqueued on the stream without waiting,
  2. enqueues the next epoch: every resident job with steps left to plan
     advances by min(remaining, epoch_steps) steps in one persistent launch
     (jobs admitted at this boundary run alongside jobs that are half done);
     with epoch_cell_steps set, epoch_steps follows the resident work so that
     an epoch stays about that many cell-steps long.  Right behind it on the
     stream goes the read-back of the observables of the jobs that this
     epoch finishes (a ticket, copied into pinned memory),
  3. retires the epoch before (with overlap on, the default): waits for its
     ticket only, so the epoch just enqueued keeps the GPU busy while the
     host hands out results, frees replicas (stream-ordered) and admits new
     jobs.  With overlap off it waits for the epoch it has just enqueued.

GPU-busy time is the sum of the epochs' durations (CUDA events around each
launch), reported per wall second and per second of the time the server had
work outstanding (the host time inside step()).  Latency is reported over finished jobs and, separately, over every
job that arrived: an unfinished job counts with the time it has waited so
far, so those percentiles are lower bounds whenever a job is censored.

A job's result does not depend on what else shares the batch (each replica
advances exactly as it would alone), which tests/test_gpu_serve.py checks.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque

import numpy as np

from . import _capi
from .batch import Batch
from .lattice import params


@dataclasses.dataclass
class Job:
    T: float
    P: float
    L: int
    sweeps: int
    seed: int
    q: int = 6
    arrival: float = 0.0          # seconds from the start of the trace
    keep_state: bool = False
    # filled by the server
    id: int = -1
    admitted: float | None = None
    finished: float | None = None
    planned: int = 0              # steps enqueued so far
    done: int = 0                 # steps completed and read back
    read_enqueued: bool = False   # its results' read-back is on the stream
    cancelled: bool = False
    error: str | None = None      # why the server refused the job
    observables: dict | None = None
    state: np.ndarray | None = None

    def cvf(self):
        return params(self.T, self.P, L=self.L, q=self.q, seed=self.seed)

    @property
    def device_bytes(self) -> int:
        # state pair + control block, tables, FP64 parameters and a small ring
        return 4 * self.L * self.L + (1 << 17)

    @property
    def latency(self) -> float | None:
        return None if self.finished is None else self.finished - self.arrival


@dataclasses.dataclass
class _Epoch:
    plan: dict            # replica id -> steps
    jobs: dict            # replica id -> job (as at enqueue time)
    finishing: list       # replica ids whose job ends with this epoch
    ticket: int           # observables of `finishing` + the launch error word
    start: object         # CUDA events around the launch
    end: object


class Server:
    """Continuous batching of jobs on one GPU."""

    def __init__(self, epoch_steps: int = 200, max_resident: int = 512,
                 hbm_reserve_bytes: int = 1 << 30, mem_budget_bytes: int | None = None,
                 tile_config: int | None = None, stream=None,
                 epoch_cell_steps: float | None = None, max_resident_cells: int | None = None,
                 overlap: bool = True):
        import torch
        self.torch = torch
        self.epoch_steps = int(epoch_steps)
        self.epoch_cell_steps = epoch_cell_steps
        self.max_resident_cells = max_resident_cells
        self.overlap = bool(overlap)
        self.resident_cells = 0
        self.max_resident = int(max_resident)
        self.reserve = int(hbm_reserve_bytes)
        self.budget = mem_budget_bytes          # optional cap on what jobs may hold
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.batch = Batch([], stream=self.stream)
        if tile_config is not None:
            self.batch.set_tiles(tile_config)
        self.total_bytes = torch.cuda.mem_get_info()[1]
        self.waiting: deque[Job] = deque()
        self.resident: dict[int, Job] = {}      # replica id -> job
        self.inflight: deque[_Epoch] = deque()
        self.finished: list[Job] = []
        self.rejected: list[Job] = []
        self.t0 = time.perf_counter()
        self.held_bytes = 0
        self.epochs = 0
        self.gpu_busy_s = 0.0                   # summed epoch durations
        self.active_s = 0.0                     # wall time inside step() / drain()
        self.steps_done = 0                     # replica steps over all jobs
        self.cell_steps = 0                     # cells x steps over all jobs
        self.queue_len: list[int] = []
        self._next_id = 0

    # --------------------------------------------------------------- intake --
    def now(self) -> float:
        return time.perf_counter() - self.t0

    def _never_fits(self, job: Job) -> str | None:
        if job.sweeps < 0:
            return "negative step count"
        cap = self.budget if self.budget is not None else self.total_bytes - self.reserve
        if job.device_bytes > cap:
            return "needs %d bytes, more than the server can ever hold (%d)" % (job.device_bytes, cap)
        return None

    def submit(self, job: Job) -> int:
        """Queues a job; a job that could not run even on an empty server is
        refused at once (job.error says why, and it goes to `rejected`)."""
        job.id = self._next_id
        self._next_id += 1
        why = self._never_fits(job)
        if why is not None:
            job.error = why
            self.rejected.append(job)
        else:
            self.waiting.append(job)
        return job.id

    def _release(self, rid: int, job: Job) -> None:
        self.batch.remove(rid)                  # stream-ordered: no wait
        self.held_bytes -= job.device_bytes
        self.resident_cells -= job.L * job.L
        del self.resident[rid]

    def cancel(self, job_id: int) -> bool:
        for j in list(self.waiting):
            if j.id == job_id:
                self.waiting.remove(j)
                j.cancelled = True
                return True
        for rid, j in list(self.resident.items()):
            if j.id == job_id:
                # epochs in flight still step it; their records of it are dropped
                j.cancelled = True
                self._release(rid, j)
                return True
        return False

    def _fits(self, job: Job) -> bool:
        if len(self.resident) >= self.max_resident:
            return False
        if (self.max_resident_cells is not None and self.resident
                and self.resident_cells + job.L * job.L > self.max_resident_cells):
            return False
        if self.budget is not None:
            return self.held_bytes + job.device_bytes <= self.budget
        free, _ = self.torch.cuda.mem_get_info()
        mapped, used = self.batch.pool_bytes()   # freed replicas stay mapped in the pool
        return free + (mapped - used) - job.device_bytes >= self.reserve

    def _admit(self) -> None:
        while self.waiting and self._fits(self.waiting[0]):
            job = self.waiting.popleft()
            rid = self.batch.add(job.cvf())
            job.admitted = self.now()
            self.resident[rid] = job
            self.held_bytes += job.device_bytes
            self.resident_cells += job.L * job.L

    # ----------------------------------------------------------------- epoch --
    def _launch(self) -> bool:
        """Enqueues the next epoch and its read-back; False if no resident
        job has steps left to plan."""
        todo = {rid: j for rid, j in self.resident.items() if j.planned < j.sweeps}
        # zero-step jobs only need their initial state read back
        idle = {rid: j for rid, j in self.resident.items()
                if j.sweeps == 0 and not j.read_enqueued}
        if not todo and not idle:
            return False
        steps = self.epoch_steps
        if self.epoch_cell_steps:
            steps = max(1, min(self.epoch_steps, int(self.epoch_cell_steps // max(1, self.resident_cells))))
        plan = [0] * self.batch.slots()
        for rid, job in todo.items():
            plan[rid] = min(steps, job.sweeps - job.planned)
        ev0 = self.torch.cuda.Event(enable_timing=True)
        ev1 = self.torch.cuda.Event(enable_timing=True)
        ev0.record(self.stream)
        if todo:
            self.batch.sweep(plan)
        ev1.record(self.stream)
        finishing = list(idle)
        for rid, job in todo.items():
            job.planned += plan[rid]
            if job.planned >= job.sweeps:
                finishing.append(rid)
        for rid in finishing:
            self.resident[rid].read_enqueued = True
        ticket = self.batch.observables_enqueue(finishing)
        self.inflight.append(_Epoch({rid: plan[rid] for rid in todo}, {**todo, **idle}, finishing,
                                    ticket, ev0, ev1))
        self.epochs += 1
        return True

    def _retire(self, ep: _Epoch) -> int:
        obs = self.batch.observables_collect(ep.ticket, len(ep.finishing))
        self.gpu_busy_s += ep.start.elapsed_time(ep.end) / 1e3
        for rid, steps in ep.plan.items():
            job = ep.jobs[rid]
            if job.cancelled:
                continue
            job.done += steps
            self.steps_done += steps
            self.cell_steps += steps * job.L * job.L
        n = 0
        for rid, o in zip(ep.finishing, obs):
            job = ep.jobs[rid]
            if job.cancelled:
                continue
            job.observables = o
            if job.keep_state:
                job.state = self.batch.state(rid)   # a zero-step replica: same lattice
            job.finished = self.now()
            self._release(rid, job)
            self.finished.append(job)
            n += 1
        return n

    def step(self) -> int:
        """Admits, enqueues one epoch and retires the one before it (or, with
        overlap off or nothing left to enqueue, everything in flight);
        returns the number of jobs that finished."""
        t0 = time.perf_counter()
        try:
            return self._step()
        finally:
            self.active_s += time.perf_counter() - t0

    def _step(self) -> int:
        self._admit()
        self.queue_len.append(len(self.waiting))
        launched = self._launch()
        keep = 1 if (launched and self.overlap) else 0
        finished = 0
        while len(self.inflight) > keep:
            finished += self._retire(self.inflight.popleft())
        return finished

    def drain(self) -> int:
        """Retires every epoch in flight."""
        t0 = time.perf_counter()
        finished = 0
        while self.inflight:
            finished += self._retire(self.inflight.popleft())
        self.active_s += time.perf_counter() - t0
        return finished

    def busy(self) -> bool:
        return bool(self.waiting or self.resident or self.inflight)

    # ------------------------------------------------------------ trace mode --
    def run_trace(self, jobs, time_limit: float | None = None) -> dict:
        """Feed jobs at their arrival times (seconds after start) and serve
        until all are done or time_limit passes; returns summary statistics."""
        pending = deque(sorted(jobs, key=lambda j: j.arrival))
        self.t0 = time.perf_counter()
        self.arrived: list[Job] = []
        while pending or self.busy():
            t = self.now()
            if time_limit is not None and t > time_limit:
                break
            while pending and pending[0].arrival <= t:
                job = pending.popleft()
                self.arrived.append(job)
                self.submit(job)
            if not self.busy():
                time.sleep(max(0.0, min(0.001, pending[0].arrival - t)) if pending else 0)
                continue
            self.step()
        self.drain()
        return self.summary(unserved=len(pending))

    def summary(self, unserved: int = 0) -> dict:
        wall = self.now()
        lat = np.array([j.latency for j in self.finished], dtype=np.float64)
        arrived = getattr(self, "arrived", None)
        if arrived is None:
            arrived = self.finished + list(self.resident.values()) + list(self.waiting)
        served = [j for j in arrived if j.error is None and not j.cancelled]
        # unfinished jobs enter with the time they have waited so far (a lower bound)
        lat_all = np.array([j.latency if j.finished is not None else wall - j.arrival
                            for j in served], dtype=np.float64)
        censored = sum(1 for j in served if j.finished is None)

        def pct(a, q):
            return float(np.percentile(a, q)) if a.size else None

        return {
            "jobs_arrived": len(arrived),
            "jobs_finished": len(self.finished),
            "jobs_resident": len(self.resident),
            "jobs_waiting": len(self.waiting) + unserved,
            "jobs_rejected": len(self.rejected),
            "jobs_censored": censored,
            "wall_s": wall,
            "epochs": self.epochs,
            "overlap": self.overlap,
            "gpu_busy_s": self.gpu_busy_s,
            "gpu_busy_per_wall_s": self.gpu_busy_s / wall if wall > 0 else 0.0,
            # the same over the wall time the server had work outstanding
            # (1.0: no host gap between epochs)
            "active_s": self.active_s,
            "gpu_busy_per_active_s": self.gpu_busy_s / self.active_s if self.active_s > 0 else 0.0,
            "replica_sweeps_per_s": self.steps_done / wall if wall > 0 else 0.0,
            "updates_per_ns": 4.0 * self.cell_steps / (wall * 1e9) if wall > 0 else 0.0,
            "latency_p50_s": pct(lat, 50),
            "latency_p99_s": pct(lat, 99),
            "latency_all_p50_s": pct(lat_all, 50),
            "latency_all_p99_s": pct(lat_all, 99),
            "latency_all_is_lower_bound": censored > 0,
            "max_queue": max(self.queue_len) if self.queue_len else 0,
        }

    def close(self) -> None:
        try:
            self.drain()
        finally:
            self.batch.close()
