"""The synthetic workload recipes have the shapes their configurations state:
the 4096^2 lattices at three temperatures and both inits, the batched
workload's 16 x 16 (T, P) grid over 270-330 K x 0.1-50 MPa with sizes from
{32 ... 512}, and the served jobs' Poisson arrivals, uniform sizes and
log-uniform step counts (CPU only)."""
import numpy as np

from paper_2505_05919_gb300 import workloads


def test_benchmark_lattices():
    c = workloads.c3()
    assert len(c) == 6 and {x["L"] for x in c} == {4096}
    assert sorted((x["init"], x["T"]) for x in c) == [(i, T) for i in (0, 1) for T in (270.0, 300.0, 330.0)]
    assert all(x["P"] == 0.1 and x["sweeps"] == 1000 and x["q"] == 6 for x in c)
    assert workloads.c1()["L"] == 64 and workloads.c2()["record_every"] == 10


def test_batched_grid_covers_the_window_once():
    c = workloads.c4()
    assert len(c) == 256
    grid = {(round(x["T"], 6), round(x["P"], 6)) for x in c}
    assert len(grid) == 256
    T = sorted({x["T"] for x in c})
    P = sorted({x["P"] for x in c})
    assert len(T) == 16 and T[0] == 270.0 and T[-1] == 330.0
    assert len(P) == 16 and P[0] == 0.1 and abs(P[-1] - 50.0) < 1e-9
    assert np.allclose(np.diff(T), 4.0) and np.allclose(np.diff(P), 49.9 / 15)
    assert {x["L"] for x in c} == {32, 64, 128, 256, 512}
    assert sorted(x["seed"] for x in c) == list(range(1000, 1256))


def test_served_jobs_distributions():
    jobs = workloads.c5(n_jobs=20000, rate_hz=200.0)
    t = np.array([j["arrival"] for j in jobs])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 200.0) < 0.05 / 200.0              # Poisson at 200/s
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05                 # exponential gaps
    L = np.array([j["L"] for j in jobs])
    counts = np.array([(L == s).sum() for s in (64, 128, 256, 512, 1024, 2048)])
    assert counts.sum() == len(jobs) and counts.min() > 0.9 * len(jobs) / 6
    sw = np.array([j["sweeps"] for j in jobs])
    assert sw.min() >= 999 and sw.max() <= 100000
    logs = np.log10(sw)
    assert abs(np.median(logs) - 4.0) < 0.05                          # log-uniform over 1e3..1e5
    T = np.array([j["T"] for j in jobs])
    P = np.array([j["P"] for j in jobs])
    assert T.min() >= 270 and T.max() <= 330 and P.min() >= 0.1 and P.max() <= 50
