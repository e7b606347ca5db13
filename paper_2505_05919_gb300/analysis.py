"""Order parameter and its autocorrelation (Sec. III.A, Eq. correlation).

M = max_q' N_q' / (number of sigma variables): the fraction of bonding
indices in the most populated state (N_q' comes from the GPU path, recorded
with the observables).  The paper normalises by qN in 3D, where the number
of sigma variables per molecule equals q = 6; on the 2D lattice there are
four per molecule, so M = max N_q' / (4N) keeps M = 1 for full order.

C_M(dt) = (<M(t0 + dt) M(t0)> - <M>^2) / (<M^2> - <M>^2), averaged over t0;
tau is the time at which C_M first reaches 1/e (linear interpolation between
the recorded lags).  These are post-processing of a recorded series.
"""
from __future__ import annotations

import math

import numpy as np

ARMS_2D = 4


def order_parameter(n_state, n_cells: int, arms: int = ARMS_2D) -> float:
    n = np.asarray(n_state, dtype=np.float64)
    return float(n.max() / (arms * n_cells))


def order_series(records, n_cells: int, arms: int = ARMS_2D) -> np.ndarray:
    return np.array([order_parameter(r["n_state"], n_cells, arms) for r in records])


def autocorrelation(series, max_lag: int | None = None) -> np.ndarray:
    """C(dt) for dt = 0..max_lag of Eq. (correlation), with <.> the average
    over all time origins available at each lag."""
    m = np.asarray(series, dtype=np.float64)
    n = m.size
    if max_lag is None:
        max_lag = n // 2
    max_lag = min(max_lag, n - 1)
    mean = m.mean()
    var = (m * m).mean() - mean * mean
    out = np.empty(max_lag + 1)
    for dt in range(max_lag + 1):
        out[dt] = ((m[dt:] * m[:n - dt]).mean() - mean * mean) / var if var > 0 else np.nan
    return out


def correlation_time(c, dt_unit: float = 1.0) -> float:
    """First lag at which C falls to 1/e, linearly interpolated (inf if never)."""
    c = np.asarray(c, dtype=np.float64)
    thr = math.exp(-1.0)
    for i in range(1, c.size):
        if c[i] <= thr:
            c0, c1 = c[i - 1], c[i]
            frac = (c0 - thr) / (c0 - c1) if c0 != c1 else 0.0
            return (i - 1 + frac) * dt_unit
    return math.inf
