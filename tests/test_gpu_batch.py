"""Batched replicas (one persistent launch) vs the same replicas run alone.

Every replica of a batch must end bit-identical (lattice, int64 counters, FP64
observables) to the single-lattice path run on its own, for every tile
configuration, with uneven lattice sizes and step counts, across several
calls, and with replicas added and removed between calls.  A few replicas are
also checked against the CPU oracle directly.
"""
from dataclasses import asdict

import numpy as np
import pytest

import oracle
from paper_2505_05919_gb300 import Batch, Lattice, params_from_dict, tile_configs, _capi
from paper_2505_05919_gb300 import autotune

pytestmark = pytest.mark.gpu

INT_KEYS = ("sweep", "n_hb", "n_hb_raw", "n_coop", "acc_sigma", "acc_volume", "g")
FP_KEYS = ("V_iso", "V", "U_LJ", "H")


def _params(L, T=300.0, P=0.1, **kw):
    return params_from_dict(asdict(oracle.physical_params(T, P, L=L, **kw)))


def _solo(p, steps_list):
    with Lattice(p) as lat:
        for n in steps_list:
            lat.sweep(n)
        return lat.state(), lat.observables()


def _same(o1, o2):
    for k in INT_KEYS:
        assert o1[k] == o2[k], k
    assert list(o1["n_state"]) == list(o2["n_state"])
    for k in FP_KEYS:
        assert abs(o1[k] - o2[k]) <= 1e-12 * abs(o2[k]), k


MIX = [  # L, T, P, extra
    (32, 270.0, 0.1, dict(seed=11)),
    (64, 300.0, 10.0, dict(seed=12, init=oracle.INIT_ORDERED)),
    (130, 330.0, 50.0, dict(seed=13)),
    (6, 300.0, 0.1, dict(seed=14, q=3)),
    (96, 285.0, 25.0, dict(seed=15, q=8)),
    (258, 300.0, 0.1, dict(seed=16)),
    (2, 300.0, 0.1, dict(seed=17)),
    (40, 3000.0, 0.1, dict(seed=18, v_iso_init=1.95, dv_max_frac=0.05)),
]


@pytest.mark.parametrize("cfg", range(12))
def test_batch_equals_solo_every_tile_config(cfg):
    ps = [_params(L, T, P, **kw) for (L, T, P, kw) in MIX]
    steps = [23, 7, 15, 40, 3, 11, 60, 33]
    with Batch(ps) as b:
        b.set_tiles(cfg)
        b.sweep(steps)
        got = [(b.state(i), b.observables(i)) for i in range(len(ps))]
    for i, p in enumerate(ps):
        s, o = _solo(p, [steps[i]])
        assert np.array_equal(got[i][0], s), (cfg, i)
        _same(got[i][1], o)


def test_batch_calls_add_remove():
    ps = [_params(L, T, P, **kw) for (L, T, P, kw) in MIX[:5]]
    with Batch(ps) as b:
        b.sweep([5, 0, 9, 2, 4])
        b.sweep([1, 6, 0, 3, 4])
        b.remove(1)
        extra = _params(48, 310.0, 5.0, seed=99)
        rid = b.add(extra)
        assert rid == 1  # the freed slot is reused
        b.sweep([2, 8, 1, 0, 4])
        res = {i: (b.state(i), b.observables(i)) for i in range(5)}
    plan = {0: [5, 1, 2], 2: [9, 0, 1], 3: [2, 3, 0], 4: [4, 4, 4]}
    for i, steps in plan.items():
        s, o = _solo(ps[i], steps)
        assert np.array_equal(res[i][0], s), i
        _same(res[i][1], o)
    s, o = _solo(extra, [8])
    assert np.array_equal(res[1][0], s)
    _same(res[1][1], o)


def test_batch_against_oracle():
    ops = [oracle.physical_params(300.0, 0.1, L=16, seed=5),
           oracle.physical_params(270.0, 20.0, L=24, seed=6, q=4),
           oracle.OracleParams(L=4, kT=3.0, P=1.2, epsilon=0.0, v_iso_init=1.9, dv_max_frac=0.2, seed=31)]
    steps = [50, 30, 200]
    with Batch([params_from_dict(asdict(o)) for o in ops]) as b:
        b.sweep(steps)
        got = [(b.state(i), b.observables(i)) for i in range(len(ops))]
    for i, op in enumerate(ops):
        ref = oracle.Oracle(op)
        ref.run(steps[i])
        assert np.array_equal(got[i][0], ref.state())
        _same(got[i][1], ref.observables())


def test_batch_many_replicas_uneven_sizes():
    rng = np.random.default_rng(4)
    Ls = rng.choice([32, 64, 128, 256], size=40)
    ps = [_params(int(L), 270.0 + 4 * (i % 16), 0.1 + (i // 16) * 3.3, seed=1000 + i)
          for i, L in enumerate(Ls)]
    with Batch(ps) as b:
        b.sweep([12] * len(ps))
        pick = [0, 7, 19, 39]
        got = {i: (b.state(i), b.observables(i)) for i in pick}
    for i in pick:
        s, o = _solo(ps[i], [12])
        assert np.array_equal(got[i][0], s)
        _same(got[i][1], o)


def test_batch_errors():
    ps = [_params(16, seed=1), _params(32, seed=2)]
    with Batch(ps) as b:
        with pytest.raises(_capi.CvfError):
            b.sweep([1])            # wrong length
        with pytest.raises(_capi.CvfError):
            b.sweep([1, -1])
        with pytest.raises(_capi.CvfError):
            b.observables(5)
        with pytest.raises(_capi.CvfError):
            b.add(_params(16, seed=3, rng_words=2))  # rng_words must match
        with pytest.raises(_capi.CvfError):
            b.add(_params(16, seed=3, schedule=oracle.SCHED_LAYERED))
        b.sweep([0, 0])
        assert b.observables(0)["sweep"] == 0


def test_autotuner_picks_a_config():
    ps = [_params(L, seed=i) for i, L in enumerate([32, 64, 128, 256])]
    best, timings = autotune.autotune(ps, probe_sweeps=5)
    assert best in timings and len(timings) == len(tile_configs())
    assert all(t > 0 for t in timings.values())


def test_batch_automatic_tile_choice():
    """The default tile setting picks, per call, the largest shape whose tiles
    over the advanced replicas still give every co-resident block a tile;
    results equal those of any fixed shape."""
    # 512 + 512 + 128 + 512 tiles of 64 x 64 words: more than the blocks
    big = [_params(L, 300.0, 0.1, seed=40 + i) for i, L in enumerate((2048, 2048, 1024, 2048))]
    small = [_params(L, 300.0, 0.1, seed=60 + i) for i, L in enumerate((32, 64, 16))]
    with Batch(big) as b:
        assert b.tiles() == (-1, -1)
        b.sweep([4] * len(big))
        assert b.tiles()[1] == 0                  # 64 x 64 words: enough tiles
        s_auto = [b.state(i) for i in range(len(big))]
    with Batch(big) as b:
        b.set_tiles(1)
        b.sweep([4] * len(big))
        assert b.tiles() == (1, 1)
        assert all(np.array_equal(b.state(i), s_auto[i]) for i in range(len(big)))
    with Batch(small) as b:
        b.sweep([4] * len(small))
        # 2 + 8 + 1 tiles of 16 x 16 words, under a quarter of the blocks:
        # the smallest tile with 512-thread blocks
        assert b.tiles()[1] == 11
        for i, p in enumerate(small):
            s, _ = _solo(p, [4])
            assert np.array_equal(b.state(i), s)
        with pytest.raises(_capi.CvfError):
            b.set_tiles(len(tile_configs()))
        b.set_tiles(-1)
        assert b.tiles()[0] == -1


def test_batch_tickets_and_stream_ordered_churn():
    """Observables read in two halves (enqueue now, collect later) describe
    the replica at the point of the stream where they were enqueued, even
    with sweeps, a removal and an add (all enqueued without waiting) behind
    them; the freed slot's memory comes back from the batch's pool."""
    ps = [_params(L, T, P, **kw) for (L, T, P, kw) in MIX[:3]]
    extra = _params(56, 305.0, 3.0, seed=77)
    with Batch(ps) as b:
        b.sweep([5, 7, 3])
        t1 = b.observables_enqueue([0, 1, 2])
        b.sweep([4, 0, 6])
        t2 = b.observables_enqueue([2])
        b.remove(1)
        assert b.add(extra) == 1
        b.sweep([0, 9, 0])
        t3 = b.observables_enqueue([1, 0])
        mapped, used = b.pool_bytes()
        assert mapped >= used > 0
        o3 = b.observables_collect(t3, 2)
        o1 = b.observables_collect(t1, 3)
        o2 = b.observables_collect(t2, 1)
        with pytest.raises(_capi.CvfError):
            b.observables_collect(t1, 2)          # wrong record count
        many = b.observables_many([0, 2, 1])
        single = [b.observables(i) for i in (0, 2, 1)]
        for a, c in zip(many, single):
            _same(a, c)
        for _ in range(4):                        # four newer tickets reuse t3's slot
            b.observables_enqueue([0])
        with pytest.raises(_capi.CvfError):
            b.observables_collect(t3, 2)
        assert b.observables_enqueue([]) >= 0
    _same(o1[0], _solo(ps[0], [5])[1])
    _same(o1[1], _solo(ps[1], [7])[1])
    _same(o1[2], _solo(ps[2], [3])[1])
    _same(o2[0], _solo(ps[2], [3, 6])[1])
    _same(o3[0], _solo(extra, [9])[1])
    _same(o3[1], _solo(ps[0], [5, 4])[1])


@pytest.mark.parametrize("cfg", [0, 3, 4, 7, 8, 11])
def test_batch_two_word_draws_every_block_size(cfg):
    """Two Philox words per update (rng_words=2) through the 256-, 128- and
    512-thread kernels."""
    mix = [(48, 290.0, 5.0, dict(seed=21)), (130, 315.0, 30.0, dict(seed=22, q=5)),
           (8, 300.0, 0.1, dict(seed=23, init=oracle.INIT_ORDERED))]
    ps = [_params(L, T, P, rng_words=2, **kw) for (L, T, P, kw) in mix]
    steps = [17, 9, 31]
    with Batch(ps) as b:
        b.set_tiles(cfg)
        b.sweep(steps)
        got = [(b.state(i), b.observables(i)) for i in range(len(ps))]
    for i, p in enumerate(ps):
        s, o = _solo(p, [steps[i]])
        assert np.array_equal(got[i][0], s), (cfg, i)
        _same(got[i][1], o)
