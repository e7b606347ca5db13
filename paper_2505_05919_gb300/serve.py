"""Continuous-batching request loop for equation-of-state scan jobs.

Jobs (a state point (T, P), a lattice side L, a number of MC steps, a seed)
arrive over time.  The server keeps every admitted job's lattice resident on
the device as one replica of a Batch.  Each epoch it

  1. admits waiting jobs in arrival order while free HBM (minus a reserve)
     covers the new replica and a slot is free,
  2. advances every resident job by min(remaining, epoch_steps) steps in one
     persistent launch (jobs admitted at this boundary run alongside jobs
     that are half done); with epoch_cell_steps set, epoch_steps follows the
     resident work so that an epoch stays about that many cell-steps long,
  3. retires finished jobs: their observables (and optionally the lattice)
     are read back and their replica is freed.

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
    done: int = 0
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


class Server:
    """Continuous batching of jobs on one GPU."""

    def __init__(self, epoch_steps: int = 200, max_resident: int = 512,
                 hbm_reserve_bytes: int = 1 << 30, mem_budget_bytes: int | None = None,
                 tile_config: int | None = None, stream=None,
                 epoch_cell_steps: float | None = None, max_resident_cells: int | None = None):
        import torch
        self.torch = torch
        self.epoch_steps = int(epoch_steps)
        self.epoch_cell_steps = epoch_cell_steps
        self.max_resident_cells = max_resident_cells
        self.resident_cells = 0
        self.max_resident = int(max_resident)
        self.reserve = int(hbm_reserve_bytes)
        self.budget = mem_budget_bytes          # optional cap on what jobs may hold
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.batch = Batch([], stream=self.stream)
        if tile_config is not None:
            self.batch.set_tiles(tile_config)
        self.waiting: deque[Job] = deque()
        self.resident: dict[int, Job] = {}      # replica id -> job
        self.finished: list[Job] = []
        self.t0 = time.perf_counter()
        self.held_bytes = 0
        self.epochs = 0
        self.steps_done = 0                     # replica steps over all jobs
        self.cell_steps = 0                     # cells x steps over all jobs
        self.queue_len: list[int] = []
        self._next_id = 0

    # --------------------------------------------------------------- intake --
    def now(self) -> float:
        return time.perf_counter() - self.t0

    def submit(self, job: Job) -> int:
        job.id = self._next_id
        self._next_id += 1
        self.waiting.append(job)
        return job.id

    def cancel(self, job_id: int) -> bool:
        for j in list(self.waiting):
            if j.id == job_id:
                self.waiting.remove(j)
                return True
        for rid, j in list(self.resident.items()):
            if j.id == job_id:
                self.batch.remove(rid)
                self.held_bytes -= j.device_bytes
                self.resident_cells -= j.L * j.L
                del self.resident[rid]
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
        return free - job.device_bytes >= self.reserve

    def _admit(self) -> None:
        while self.waiting and self._fits(self.waiting[0]):
            job = self.waiting.popleft()
            rid = self.batch.add(job.cvf())
            job.admitted = self.now()
            self.resident[rid] = job
            self.held_bytes += job.device_bytes
            self.resident_cells += job.L * job.L

    # ----------------------------------------------------------------- epoch --
    def step(self) -> int:
        """One epoch; returns the number of jobs that finished in it."""
        self._admit()
        self.queue_len.append(len(self.waiting))
        if not self.resident:
            return 0
        n = self.batch.slots()
        steps = self.epoch_steps
        if self.epoch_cell_steps:
            steps = max(1, min(self.epoch_steps, int(self.epoch_cell_steps // max(1, self.resident_cells))))
        plan = [0] * n
        for rid, job in self.resident.items():
            plan[rid] = min(steps, job.sweeps - job.done)
        self.batch.sweep(plan)
        self.batch.sync()
        self.epochs += 1
        finished = 0
        for rid, job in list(self.resident.items()):
            job.done += plan[rid]
            self.steps_done += plan[rid]
            self.cell_steps += plan[rid] * job.L * job.L
            if job.done >= job.sweeps:
                job.observables = self.batch.observables(rid)
                if job.keep_state:
                    job.state = self.batch.state(rid)
                job.finished = self.now()
                self.batch.remove(rid)
                self.held_bytes -= job.device_bytes
                self.resident_cells -= job.L * job.L
                del self.resident[rid]
                self.finished.append(job)
                finished += 1
        return finished

    def busy(self) -> bool:
        return bool(self.waiting or self.resident)

    # ------------------------------------------------------------ trace mode --
    def run_trace(self, jobs, time_limit: float | None = None) -> dict:
        """Feed jobs at their arrival times (seconds after start) and serve
        until all are done or time_limit passes; returns summary statistics."""
        pending = deque(sorted(jobs, key=lambda j: j.arrival))
        self.t0 = time.perf_counter()
        while pending or self.busy():
            t = self.now()
            if time_limit is not None and t > time_limit:
                break
            while pending and pending[0].arrival <= t:
                self.submit(pending.popleft())
            if not self.busy():
                time.sleep(max(0.0, min(0.001, pending[0].arrival - t)) if pending else 0)
                continue
            self.step()
        return self.summary(unserved=len(pending))

    def summary(self, unserved: int = 0) -> dict:
        wall = self.now()
        lat = np.array([j.latency for j in self.finished], dtype=np.float64)
        return {
            "jobs_finished": len(self.finished),
            "jobs_resident": len(self.resident),
            "jobs_waiting": len(self.waiting) + unserved,
            "wall_s": wall,
            "epochs": self.epochs,
            "replica_sweeps_per_s": self.steps_done / wall if wall > 0 else 0.0,
            "updates_per_ns": 4.0 * self.cell_steps / (wall * 1e9) if wall > 0 else 0.0,
            "latency_p50_s": float(np.percentile(lat, 50)) if lat.size else None,
            "latency_p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "max_queue": max(self.queue_len) if self.queue_len else 0,
        }

    def close(self) -> None:
        self.batch.close()
