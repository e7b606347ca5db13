"""The autotuner's search and cache on the CPU: every configuration is
probed on a scratch batch (other seeds than the caller's replicas), the
fastest is returned, and the result is cached by the lattice-size mix and
probe length (not by the state points).  The batch and the CUDA events are
fakes whose "time" per step is a fixed cost per configuration."""
import pytest
import torch

from paper_2505_05919_gb300 import autotune as AT
from paper_2505_05919_gb300 import params
from paper_2505_05919_gb300.batch import tile_configs

COST = {}   # configuration -> ms per step of the fake batch


class FakeBatch:
    made = []

    def __init__(self, params_list=(), stream=None):
        self.params = list(params_list)
        self.cfg = None
        self.steps = 0
        FakeBatch.made.append(self)

    def slots(self):
        return len(self.params)

    def set_tiles(self, c):
        self.cfg = c

    def sweep(self, plan):
        assert len(plan) == len(self.params)
        FakeEvent.pending = COST[self.cfg] * plan[0]

    def sync(self):
        pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


class FakeEvent:
    pending = 0.0
    clock = 0.0

    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        FakeEvent.clock += FakeEvent.pending
        FakeEvent.pending = 0.0
        self.t = FakeEvent.clock

    def synchronize(self):
        pass

    def elapsed_time(self, other):
        return other.t - self.t


@pytest.fixture
def fakes(monkeypatch):
    AT._cache.clear()
    FakeBatch.made.clear()
    monkeypatch.setattr(AT, "Batch", FakeBatch)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "Stream", lambda *a, **k: object())
    n = len(tile_configs())
    COST.clear()
    COST.update({c: 1.0 + 0.1 * c for c in range(n)})
    yield
    AT._cache.clear()


def reps(T=300.0, P=0.1, sizes=(32, 64, 128)):
    return [params(T, P, L=L, q=6, seed=10 + i) for i, L in enumerate(sizes)]


def test_the_fastest_configuration_is_returned_with_every_timing(fakes):
    COST[5] = 0.25
    best, t = AT.autotune(reps(), probe_sweeps=20)
    assert best == 5
    assert set(t) == set(range(len(tile_configs())))
    assert t[5] == pytest.approx(0.25) and t[0] == pytest.approx(1.0)


def test_the_probe_runs_on_scratch_replicas_of_the_same_sizes(fakes):
    ps = reps()
    AT.autotune(ps, probe_sweeps=20)
    scratch = FakeBatch.made[-1].params
    assert [p.L for p in scratch] == [p.L for p in ps]
    assert all(s.seed != p.seed for s, p in zip(scratch, ps))
    assert [p.seed for p in ps] == [10, 11, 12]      # the caller's replicas untouched


def test_cached_by_size_mix_and_probe_length_not_by_state_point(fakes):
    COST[3] = 0.5
    best, _ = AT.autotune(reps(270.0, 0.1), probe_sweeps=20)
    assert best == 3 and len(FakeBatch.made) == 1
    COST[3] = 9.0   # a second probe would now pick another configuration
    assert AT.autotune(reps(330.0, 50.0), probe_sweeps=20)[0] == 3   # same sizes: cached
    assert AT.autotune(list(reversed(reps())), probe_sweeps=20)[0] == 3  # order does not matter
    assert len(FakeBatch.made) == 1
    assert AT.autotune(reps(), probe_sweeps=10)[0] != 3                  # another probe length
    assert AT.autotune(reps(sizes=(32, 64, 256)), probe_sweeps=20)[0] != 3  # another mix
    assert len(FakeBatch.made) == 3


def test_cells_per_thread_follows_the_configuration():
    for c, (rows, words, threads) in enumerate(tile_configs()):
        assert AT.cells_per_thread(c) == 2 * rows * words // threads
    assert AT.cells_per_thread(0) == 32        # 64 x 64 words, 256 threads
