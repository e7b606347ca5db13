"""Order parameter M and its autocorrelation (Eq. correlation), pinned on the
CPU: the oracle's N_q' against a direct count; M's range and extremes; the
autocorrelation of an AR(1) series against its closed form rho^dt and its
1/e time -1/ln(rho); a pure cosine against cos(w dt)."""
import math

import numpy as np
import pytest

import oracle
from paper_2505_05919_gb300 import analysis


def test_oracle_state_counts_direct():
    p = oracle.OracleParams(L=12, q=5, seed=4, kT=0.5)
    o = oracle.Oracle(p)
    o.run(7)
    ob = o.observables()
    w = o.state().ravel().astype(np.int64)
    direct = np.zeros(8, np.int64)
    for a in range(4):
        direct += np.bincount((w >> (4 * a)) & 7, minlength=8)
    assert list(ob["n_state"]) == list(direct)
    assert sum(ob["n_state"]) == 4 * 144 and all(x == 0 for x in ob["n_state"][5:])


def test_order_parameter_extremes():
    N = 100
    assert analysis.order_parameter([4 * N, 0, 0, 0, 0, 0, 0, 0], N) == 1.0
    assert analysis.order_parameter([400 / 6] * 6 + [0, 0], N) == pytest.approx(1 / 6)
    p = oracle.OracleParams(L=8, q=6, init=oracle.INIT_ORDERED, kT=1e-3, volume_moves=0)
    o = oracle.Oracle(p)
    o.run(3)
    assert analysis.order_parameter(o.observables()["n_state"], 64) == 1.0


def test_autocorrelation_ar1_closed_form():
    rho, n = 0.9, 400000
    rng = np.random.default_rng(1)
    e = rng.normal(size=n)
    x = np.empty(n)
    x[0] = e[0] / math.sqrt(1 - rho * rho)
    for i in range(1, n):
        x[i] = rho * x[i - 1] + e[i]
    c = analysis.autocorrelation(x, 40)
    assert np.allclose(c, rho ** np.arange(41), atol=0.02)
    assert analysis.correlation_time(c) == pytest.approx(-1 / math.log(rho), rel=0.05)


def test_autocorrelation_cosine():
    w = 2 * math.pi / 50
    t = np.arange(50 * 400)
    c = analysis.autocorrelation(np.cos(w * t), 60)
    assert np.allclose(c, np.cos(w * np.arange(61)), atol=0.01)
    assert analysis.correlation_time(np.ones(10)) == math.inf
