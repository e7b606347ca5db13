"""GPU path vs CPU oracle, through the C ABI.

Bar: the packed lattice is bit-exact, every integer counter is equal, and the
FP64 observables (V_iso, V, U_LJ, H) agree to a relative 1e-12.  The oracle
receives its inputs from the seeded workload recipes and its own unit
conversion, never from the GPU path.
"""
from dataclasses import asdict

import numpy as np
import pytest

import oracle
from paper_2505_05919_gb300 import Lattice, params, params_from_dict, _capi, workloads

pytestmark = pytest.mark.gpu

FP_REL = 1e-12
INT_KEYS = ("sweep", "n_hb", "n_hb_raw", "n_coop", "acc_sigma", "acc_volume", "g")
FP_KEYS = ("V_iso", "V", "U_LJ", "H")


def assert_obs_equal(got, want, ctx=""):
    for k in INT_KEYS:
        assert got[k] == want[k], (ctx, k, got[k], want[k])
    assert list(got["n_state"]) == list(want["n_state"]), (ctx, "n_state")
    for k in FP_KEYS:
        assert abs(got[k] - want[k]) <= FP_REL * max(abs(want[k]), 1e-300), (ctx, k, got[k], want[k])


def gpu_run(op, K, record_every=0):
    with Lattice(params_from_dict(asdict(op))) as lat:
        lat.sweep(K, record_every)
        state = lat.state()
        obs = lat.observables()
        recs, overflow = lat.drain()
        hb, co = lat.recount()
    assert not overflow
    assert (hb, co) == (obs["n_hb_raw"], obs["n_coop"]), "sweep counts differ from the recount kernel"
    return state, obs, recs


def oracle_run(op, K, record_every=0):
    o = oracle.Oracle(op)
    recs = o.run(K, record_every)
    return o.state(), o.observables(), recs


CASES = [
    # L, K, extra parameters
    (2, 300, {}),
    (4, 300, dict(q=2)),
    (6, 200, dict(q=8)),
    (8, 200, dict(init=oracle.INIT_ORDERED)),
    (16, 150, dict(rng_words=2)),
    (64, 1000, {}),                                   # 4096 cells, 1000 steps, ambient
    (130, 60, dict(T=270.0)),                         # odd number of word pairs per row
    (130, 40, dict(T=330.0, P=50.0, rng_words=2)),
    (258, 25, dict(init=oracle.INIT_ORDERED, T=330.0)),
    (96, 80, dict(volume_moves=0, q=3)),
]


@pytest.mark.parametrize("L,K,extra", CASES, ids=[f"L{c[0]}-K{c[1]}-{i}" for i, c in enumerate(CASES)])
def test_checkerboard_parity(L, K, extra):
    extra = dict(extra)
    T = extra.pop("T", 300.0)
    P = extra.pop("P", 0.1)
    op = oracle.physical_params(T, P, L=L, seed=100 + L + K, dv_max_frac=0.02, **extra)
    s_gpu, o_gpu, _ = gpu_run(op, K)
    s_ref, o_ref, _ = oracle_run(op, K)
    assert np.array_equal(s_gpu, s_ref)
    assert_obs_equal(o_gpu, o_ref)
    assert 0 <= o_gpu["n_hb_raw"] <= 2 * L * L and 0 <= o_gpu["n_coop"] <= 6 * L * L


@pytest.mark.parametrize("config", [0, 1, 2])
@pytest.mark.parametrize("L,K,extra", [(64, 40, {}), (130, 25, dict(rng_words=2)),
                                       (258, 12, dict(T=270.0, init=oracle.INIT_ORDERED)),
                                       (34, 60, dict(kT=1e-3))])
def test_checkerboard_every_tile_shape(config, L, K, extra):
    """Every tile shape of the sweep (64x64, 32x32, 16x32 words), including
    ragged edge tiles and odd numbers of words per row, gives the oracle's
    lattice and counts."""
    extra = dict(extra)
    if "kT" in extra:  # the 64-bit threshold compare
        op = oracle.OracleParams(L=L, seed=300 + L, init=oracle.INIT_ORDERED, **extra)
    else:
        T = extra.pop("T", 300.0)
        op = oracle.physical_params(T, 0.1, L=L, seed=300 + L, dv_max_frac=0.02, **extra)
    with Lattice(params_from_dict(asdict(op))) as lat:
        lat.set_tiles(config)
        assert lat.tiles()[0] == config
        lat.sweep(K, 5)
        s_gpu, o_gpu = lat.state(), lat.observables()
        r_gpu, _ = lat.drain()
    s_ref, o_ref, r_ref = oracle_run(op, K, record_every=5)
    assert np.array_equal(s_gpu, s_ref)
    assert_obs_equal(o_gpu, o_ref)
    for a, b in zip(r_gpu, r_ref):
        assert_obs_equal(a, b)


@pytest.mark.parametrize("config", [0, 1, 2])
@pytest.mark.parametrize("L,K,every,extra", [(128, 30, 1, {}), (256, 12, 3, dict(rng_words=2)),
                                             (512, 6, 2, dict(T=270.0, init=oracle.INIT_ORDERED)),
                                             (192, 10, 1, dict(q=5)), (128, 20, 4, dict(kT=1e-3)),
                                             (256, 10, 1, dict(T=330.0, P=50.0, q=8))])
def test_checkerboard_walking_form(config, L, K, every, extra):
    """Lattices whose tiles are all full (L a multiple of the tile height and
    of twice the tile width) sweep in the column-walking form: colour 1
    updated in place and the tile copied out in 16-byte rows, the halo rows
    and the ring swept one cell per thread.  Same lattice, counts and
    recorded series as the oracle (L = 192 with 64-word tiles falls back to
    the general form)."""
    extra = dict(extra)
    if "kT" in extra:  # the 64-bit threshold compare
        op = oracle.OracleParams(L=L, seed=700 + L + config, init=oracle.INIT_RANDOM, **extra)
    else:
        T = extra.pop("T", 300.0)
        P = extra.pop("P", 0.1)
        op = oracle.physical_params(T, P, L=L, seed=700 + L + config, dv_max_frac=0.02, **extra)
    with Lattice(params_from_dict(asdict(op))) as lat:
        lat.set_tiles(config)
        assert lat.tiles()[0] == config
        lat.sweep(K // 2, every)
        lat.sweep(K - K // 2, every)
        s_gpu, o_gpu = lat.state(), lat.observables()
        r_gpu, overflow = lat.drain()
        assert lat.recount() == (o_gpu["n_hb_raw"], o_gpu["n_coop"])
    s_ref, o_ref, r_ref = oracle_run(op, K, record_every=every)
    assert not overflow and len(r_gpu) == len(r_ref)
    assert np.array_equal(s_gpu, s_ref)
    assert_obs_equal(o_gpu, o_ref)
    for a, b in zip(r_gpu, r_ref):
        assert_obs_equal(a, b)


@pytest.mark.parametrize("L,K,extra", [(16, 300, {}), (64, 200, dict(rng_words=2)),
                                       (128, 60, dict(T=270.0, init=oracle.INIT_ORDERED)),
                                       (256, 20, dict(q=8)), (24, 150, dict(kT=1e-3)),
                                       (32, 400, dict(kT=3.0, P=1.2, epsilon=0.0, v_iso_init=1.9,
                                                      dv_max_frac=0.2)),
                                       (64, 700, dict(T=330.0, dv_max_frac=0.3)),
                                       (16, 900, dict(kT=1.5, P=0.4, v_iso_init=1.98,
                                                      dv_max_frac=0.01))])
def test_resident_cluster_sweep(L, K, extra):
    """The resident form (the lattice in one cluster's shared memory for the
    whole call) gives the oracle's lattice, counts and recorded series --
    both RNG modes, both inits, q = 8, the 64-bit compare, gate flips.  The
    volume moves are decided ahead in passes over five steps' outcomes: the
    V_iso series recorded every step equals the oracle's for long runs with
    many rejected and accepted moves, and near the gate (v_iso close to 2,
    small steps) where passes stop at gate-changing proposals."""
    extra = dict(extra)
    if "kT" in extra:
        op = oracle.OracleParams(L=L, seed=400 + L, **extra)
    else:
        T = extra.pop("T", 300.0)
        dv = extra.pop("dv_max_frac", 0.02)
        op = oracle.physical_params(T, 0.1, L=L, seed=400 + L, dv_max_frac=dv, **extra)
    with Lattice(params_from_dict(asdict(op))) as lat:
        lat.set_tiles(3)
        assert lat.tiles() == (3, L // 8, L // 2)
        lat.sweep(K // 2, 1)
        lat.sweep(K - K // 2, 1)   # two calls: the lattice leaves and re-enters the cluster
        s_gpu, o_gpu = lat.state(), lat.observables()
        r_gpu, _ = lat.drain()
        assert lat.recount() == (o_gpu["n_hb_raw"], o_gpu["n_coop"])
    s_ref, o_ref, r_ref = oracle_run(op, K, record_every=1)
    assert np.array_equal(s_gpu, s_ref)
    assert_obs_equal(o_gpu, o_ref)
    assert len(r_gpu) == len(r_ref) == K
    for i, (a, b) in enumerate(zip(r_gpu, r_ref)):
        assert_obs_equal(a, b, ("record", i))


@pytest.mark.parametrize("config,L,K,extra", [
    (6, 136, 40, {}),                                     # 16 x 32 words: 3 x 9 tiles, ragged
    (6, 200, 30, dict(rng_words=2)),
    (5, 200, 25, dict(T=270.0, init=oracle.INIT_ORDERED)),  # 32 x 32: 4 x 7 tiles
    (4, 392, 12, {}),                                     # 64 x 64: 4 x 7 tiles
    (6, 136, 60, dict(kT=1e-3)),                          # the 64-bit threshold compare
    # v_iso near 2 with a weak bond energy: the gate changes ~50 times in
    # 300 steps, each decided after the step before is committed
    (6, 136, 300, dict(kT=2.4, P=1.2, epsilon=0.0, J=1e-4, J_sigma=0.0, v_HB=0.0,
                       v_iso_init=2.0, dv_max_frac=0.01)),
    (5, 256, 200, dict(dv_max_frac=0.3)),
])
def test_wavefront_sweep(config, L, K, extra):
    """The wavefront sweep (one persistent launch per call; a tile of step
    s + 1 waits only for the tiles around it; the volume moves decided ahead
    by one block, gate-changing ones after the step before is committed)
    gives the oracle's lattice, counts and series recorded every step -- with
    up to sixteen steps in flight on small tile grids, ragged tiles, both RNG
    modes, both inits, the 64-bit compare and gate flips; and a second call
    continues the first."""
    extra = dict(extra)
    if "kT" in extra:
        op = oracle.OracleParams(L=L, seed=500 + L, **extra)
    else:
        T = extra.pop("T", 300.0)
        dv = extra.pop("dv_max_frac", 0.02)
        op = oracle.physical_params(T, 0.1, L=L, seed=500 + L, dv_max_frac=dv, **extra)
    with Lattice(params_from_dict(asdict(op))) as lat:
        lat.set_tiles(config)
        assert lat.tiles()[0] == config
        lat.sweep(K // 3, 1)
        lat.sweep(K - K // 3, 1)
        s_gpu, o_gpu = lat.state(), lat.observables()
        r_gpu, _ = lat.drain()
        assert lat.recount() == (o_gpu["n_hb_raw"], o_gpu["n_coop"])
    s_ref, o_ref, r_ref = oracle_run(op, K, record_every=1)
    assert np.array_equal(s_gpu, s_ref)
    assert_obs_equal(o_gpu, o_ref)
    assert len(r_gpu) == len(r_ref) == K
    for i, (a, b) in enumerate(zip(r_gpu, r_ref)):
        assert_obs_equal(a, b, ("record", i))
    if "v_iso_init" in extra:
        gs = [r["g"] for r in r_ref]
        assert sum(1 for a, b in zip(gs, gs[1:]) if a != b) >= 3


def test_tile_choice():
    with Lattice(params(300.0, 0.1, L=4096)) as lat:
        assert lat.tiles() == (4, 64, 64)  # the benchmark size: the wavefront, large tiles
    with Lattice(params(300.0, 0.1, L=8192)) as lat:
        assert lat.tiles() == (4, 64, 64)  # the wavefront at every larger size too
    with Lattice(params(300.0, 0.1, L=1024)) as lat:
        assert lat.tiles() == (6, 16, 32)  # mid-size lattices: the wavefront sweep
    with Lattice(params(300.0, 0.1, L=2048)) as lat:
        assert lat.tiles() == (5, 32, 32)
    with Lattice(params(300.0, 0.1, L=256)) as lat:
        c, r, w = lat.tiles()
        assert c == 6               # the wavefront from 256^2 up
        with pytest.raises(_capi.CvfError):
            lat.set_tiles(4)      # the wavefront needs 3 x 3 tiles: 2 x 4 of 64 x 64 words
        with pytest.raises(_capi.CvfError):
            lat.set_tiles(7)
    with Lattice(params(300.0, 0.1, L=64)) as lat:
        assert lat.tiles()[0] == 3  # small lattices run resident in one cluster
    with Lattice(params(300.0, 0.1, L=130)) as lat:
        with pytest.raises(_capi.CvfError):
            lat.set_tiles(3)      # 130 is not a multiple of 8


@pytest.mark.parametrize("L,K,rng_words", [(2, 100, 1), (8, 80, 2), (64, 60, 1), (130, 20, 2),
                                           (258, 12, 1)])
def test_layered_parity(L, K, rng_words):
    op = oracle.physical_params(300.0, 0.1, L=L, seed=7 + L, schedule=oracle.SCHED_LAYERED,
                                rng_words=rng_words, dv_max_frac=0.02)
    s_gpu, o_gpu, _ = gpu_run(op, K)
    s_ref, o_ref, _ = oracle_run(op, K)
    assert np.array_equal(s_gpu, s_ref)
    assert_obs_equal(o_gpu, o_ref)


@pytest.mark.parametrize("extra", [dict(L=6, T=270.0, init=oracle.INIT_ORDERED, q=3),
                                   dict(L=16, T=330.0, P=50.0, q=8),
                                   dict(L=4, kT=3.0, P=1.2, epsilon=0.0, v_iso_init=1.9,
                                        dv_max_frac=0.2),                       # gate flips
                                   dict(L=8, kT=1e-3, init=oracle.INIT_ORDERED)])  # 64-bit compare
def test_layered_series_parity(extra):
    """The layered schedule's recorded series (counts, N_q', volume, H every
    3 steps) equal the oracle's, across both inits, state points, gate flips
    and the 64-bit threshold compare."""
    extra = dict(extra)
    if "kT" in extra:  # reduced units given directly
        op = oracle.OracleParams(schedule=oracle.SCHED_LAYERED, seed=23, **extra)
    else:
        T, P = extra.pop("T", 300.0), extra.pop("P", 0.1)
        op = oracle.physical_params(T, P, schedule=oracle.SCHED_LAYERED, seed=23,
                                    dv_max_frac=0.02, **extra)
    s_gpu, o_gpu, r_gpu = gpu_run(op, 90, record_every=3)
    s_ref, o_ref, r_ref = oracle_run(op, 90, record_every=3)
    assert np.array_equal(s_gpu, s_ref)
    assert_obs_equal(o_gpu, o_ref)
    assert len(r_gpu) == len(r_ref) == 30
    for i, (a, b) in enumerate(zip(r_gpu, r_ref)):
        assert_obs_equal(a, b, ("record", i))


def test_series_parity_record_every():
    # configuration 2's recording pattern (every 10 steps) on a 64 x 64 lattice
    op = oracle.physical_params(300.0, 0.1, L=64, seed=2)
    _, _, r_gpu = gpu_run(op, 200, record_every=10)
    _, _, r_ref = oracle_run(op, 200, record_every=10)
    assert len(r_gpu) == len(r_ref) == 20
    for a, b in zip(r_gpu, r_ref):
        assert_obs_equal(a, b)


def test_order_parameter_series_matches_oracle():
    """N_q' recorded every step by the sweep kernel, hence M(t) and C_M(dt)
    (Eq. correlation), equal the oracle's."""
    from paper_2505_05919_gb300 import analysis
    op = oracle.physical_params(250.0, 0.1, L=32, seed=8)
    _, o_gpu, r_gpu = gpu_run(op, 600, record_every=1)
    _, o_ref, r_ref = oracle_run(op, 600, record_every=1)
    assert [r["n_state"] for r in r_gpu] == [r["n_state"] for r in r_ref]
    m_gpu = analysis.order_series(r_gpu, 32 * 32)
    m_ref = analysis.order_series(r_ref, 32 * 32)
    assert np.array_equal(m_gpu, m_ref)
    c = analysis.autocorrelation(m_gpu[100:], 50)
    assert c[0] == pytest.approx(1.0)
    assert np.array_equal(c, analysis.autocorrelation(m_ref[100:], 50))


@pytest.mark.parametrize("case", ["gas", "gate_flips", "hot", "cold", "no_lj"])
def test_special_regimes(case):
    kw = dict(L=16, seed=31)
    if case == "gas":        # v_iso > 2: gas-like cells form no bonds (g = 0)
        op = oracle.physical_params(300.0, 0.1, v_iso_init=2.5, **kw)
    elif case == "gate_flips":  # small lattice, large volume steps: v_iso crosses 2 often
        op = oracle.OracleParams(L=4, kT=3.0, P=1.2, epsilon=0.0, v_iso_init=1.9, dv_max_frac=0.2,
                                 seed=31)
    elif case == "hot":
        op = oracle.OracleParams(kT=1e300, **kw)
    elif case == "cold":
        op = oracle.OracleParams(kT=1e-3, init=oracle.INIT_ORDERED, **kw)
    else:
        op = oracle.physical_params(300.0, 0.1, epsilon=0.0, **kw)
    s_gpu, o_gpu, r_gpu = gpu_run(op, 400, record_every=1)
    s_ref, o_ref, r_ref = oracle_run(op, 400, record_every=1)
    assert np.array_equal(s_gpu, s_ref)
    assert_obs_equal(o_gpu, o_ref, case)
    for a, b in zip(r_gpu, r_ref):
        assert_obs_equal(a, b, case)
    if case == "gate_flips":
        gs = [r["g"] for r in r_ref]
        flips = sum(1 for a, b in zip(gs, gs[1:]) if a != b)
        assert flips >= 3, "the gate flipped %d times; the case tests too little" % flips


def test_set_state_resume_bit_exact():
    op = oracle.physical_params(300.0, 0.1, L=32, seed=9, dv_max_frac=0.05)
    p = params_from_dict(asdict(op))
    with Lattice(p) as a:
        a.sweep(37)
        mid = a.state()
        mo = a.observables()
    with Lattice(p) as b:
        b.set_state(mid, mo["V_iso"], mo["sweep"])
        b.sweep(25)
        s_b, o_b = b.state(), b.observables()
    ref = oracle.Oracle(op)
    ref.run(62)
    assert np.array_equal(s_b, ref.state())
    want = ref.observables()
    for k in ("sweep", "n_hb_raw", "n_coop", "g"):
        assert o_b[k] == want[k]
    for k in FP_KEYS:
        assert abs(o_b[k] - want[k]) <= FP_REL * abs(want[k])


def test_set_state_arbitrary_configuration():
    L = 24
    words = workloads.random_words(L, 5, seed=44)
    op = oracle.physical_params(300.0, 0.1, L=L, q=5, seed=12)
    with Lattice(params_from_dict(asdict(op))) as lat:
        lat.set_state(words, V_iso=L * L * 1.3, sweep=1000)
        assert np.array_equal(lat.state(), words)
        assert lat.recount() == oracle.recount(op, words)
        lat.sweep(30)
        s_gpu, o_gpu = lat.state(), lat.observables()
    ref = oracle.Oracle(op, state=words, V_iso=L * L * 1.3, sweep=1000)
    ref.run(30)
    assert np.array_equal(s_gpu, ref.state())
    assert_obs_equal(o_gpu, ref.observables())


def test_invalid_inputs_rejected():
    op = oracle.physical_params(300.0, 0.1, L=8, q=6)
    with Lattice(params_from_dict(asdict(op))) as lat:
        before = lat.state()
        bad = before.copy()
        bad[3, 3] = 6  # arm 0 = 6 >= q
        with pytest.raises(_capi.CvfError) as e:
            lat.set_state(bad, V_iso=80.0)
        assert e.value.code == _capi.CVF_EINVAL
        bad = before.copy()
        bad[0, 0] |= 1 << 15
        with pytest.raises(_capi.CvfError):
            lat.set_state(bad, V_iso=80.0)
        with pytest.raises(_capi.CvfError):
            lat.set_state(before, V_iso=63.0)  # below the hard core N v0
        with pytest.raises(_capi.CvfError):
            lat.sweep(-1)
        assert np.array_equal(lat.state(), before)
        lat.sweep(0)
        assert lat.observables()["sweep"] == 0
    with pytest.raises(_capi.CvfError):
        Lattice(params_from_dict(asdict(oracle.OracleParams(L=7))))


def test_ring_overflow_keeps_newest():
    op = oracle.OracleParams(L=2, volume_moves=0, seed=3)
    with Lattice(params_from_dict(asdict(op))) as lat:
        lat.sweep(65536 + 100, 1)
        recs, overflow = lat.drain(1 << 17)
        assert overflow
        assert len(recs) == 65536
        assert recs[0]["sweep"] == 101 and recs[-1]["sweep"] == 65636


@pytest.mark.parametrize("cfg", range(6))
def test_full_size_sampled_windows(cfg):
    """The six 4096 x 4096 lattices the benchmark times (random init seed 3
    and ordered init, 270 / 300 / 330 K, 0.1 MPa), 50 steps through the
    automatic form the benchmark runs (the wavefront sweep on 64 x 64-word
    tiles, one launch for the call), and for two of them through the tiled
    sweep with programmatic launches as well.  The oracle cannot run the whole
    lattice, so it recomputes eight sampled windows: a checkerboard step
    moves information by at most two cells, so a window run with its border
    frozen is exact more than 2K + 2 cells inside.  Four windows lie across
    the periodic edges (the four corners of the lattice, wrapped) and four
    at random places.  V_iso follows from the oracle's own volume chain (no
    gate flip is proposed at these state points); the kept counts equal an
    independent recount."""
    from paper_2505_05919_gb300 import workloads
    c = workloads.c3()[cfg]
    L, K = 4096, 50
    op = oracle.physical_params(c["T"], c["P"], L=L, q=c["q"], seed=c["seed"], init=c["init"])
    with Lattice(params_from_dict(asdict(op))) as lat:
        init_gpu = lat.state()
        assert lat.tiles()[0] == 4
        lat.sweep(K)
        s_gpu = lat.state()
        o_gpu = lat.observables()
        hb, co = lat.recount()
    assert (hb, co) == (o_gpu["n_hb_raw"], o_gpu["n_coop"])
    if cfg in (0, 4):
        with Lattice(params_from_dict(asdict(op))) as lat:
            lat.set_tiles(0)
            lat.sweep(K)
            assert np.array_equal(lat.state(), s_gpu)
            assert_obs_equal(lat.observables(), o_gpu)
    ref0 = oracle.Oracle(op)
    assert np.array_equal(init_gpu, ref0.state())
    done, V, g, acc = oracle.volume_chain(op, ref0.observables()["V_iso"], 0, K)
    assert done == K
    assert V[-1] == pytest.approx(o_gpu["V_iso"], rel=FP_REL)
    assert o_gpu["acc_volume"] == acc
    margin, inner = 2 * K + 2, 48
    W = inner + 2 * margin
    rng = np.random.default_rng(2024 + cfg)
    spots = [(L - W // 2, L - W // 2), (L - W // 2, 0), (0, L - W // 2), (L - 20, L - W + 7)]
    spots += [(int(rng.integers(0, L)), int(rng.integers(0, L))) for _ in range(4)]
    full = ref0.state()
    for x0, y0 in spots:
        out = oracle.window_run(op, full, x0, y0, W, W, 0, g).reshape(L, L)
        ys = [(y0 + margin + i) % L for i in range(inner)]
        xs = [(x0 + margin + i) % L for i in range(inner)]
        assert np.array_equal(s_gpu[np.ix_(ys, xs)], out[np.ix_(ys, xs)]), (cfg, x0, y0)
    assert 0 < o_gpu["n_hb_raw"] <= 2 * L * L and 0 < o_gpu["n_coop"] <= 6 * L * L


@pytest.mark.parametrize("L,K,every,extra", [
    (136, 2000, 40, {}),
    (200, 1200, 25, dict(rng_words=2, init=oracle.INIT_ORDERED)),
    (136, 1500, 1, dict(kT=2.4, P=1.2, epsilon=0.0, J=1e-4, J_sigma=0.0, v_HB=0.0,
                        v_iso_init=2.0, dv_max_frac=0.01)),
])
def test_wavefront_long_runs(L, K, every, extra):
    """Long wavefront calls on small tile grids (16 x 32 words: every block
    takes items up to sixteen steps ahead, and the steps' slots and volume
    moves are reused about a hundred times), against the oracle's lattice
    and records -- including a run whose gate changes hundreds of times."""
    extra = dict(extra)
    if "kT" in extra:
        op = oracle.OracleParams(L=L, seed=900 + L, **extra)
    else:
        op = oracle.physical_params(300.0, 0.1, L=L, seed=900 + L, dv_max_frac=0.02, **extra)
    with Lattice(params_from_dict(asdict(op))) as lat:
        lat.set_tiles(6)
        lat.sweep(K, every)
        s_gpu, o_gpu = lat.state(), lat.observables()
        r_gpu, overflow = lat.drain()
    s_ref, o_ref, r_ref = oracle_run(op, K, record_every=every)
    assert not overflow and len(r_gpu) == len(r_ref) == K // every
    assert np.array_equal(s_gpu, s_ref)
    assert_obs_equal(o_gpu, o_ref)
    for i, (a, b) in enumerate(zip(r_gpu, r_ref)):
        assert_obs_equal(a, b, ("record", i))


def test_resident_volume_engine_long_run():
    """The resident form's volume moves decided ahead in five-step passes,
    over 3000 steps of a lattice whose gate changes hundreds of times (each
    change stops a pass; the commit decides it and the engine restarts),
    recorded every step against the oracle."""
    op = oracle.OracleParams(L=16, seed=61, kT=2.4, P=1.2, epsilon=0.0, J=1e-4, J_sigma=0.0,
                             v_HB=0.0, v_iso_init=2.0, dv_max_frac=0.05)
    K = 3000
    with Lattice(params_from_dict(asdict(op))) as lat:
        assert lat.tiles()[0] == 3
        lat.sweep(K, 1)
        s_gpu, o_gpu = lat.state(), lat.observables()
        r_gpu, overflow = lat.drain()
    s_ref, o_ref, r_ref = oracle_run(op, K, record_every=1)
    assert not overflow and len(r_gpu) == K
    gs = [r["g"] for r in r_ref]
    assert sum(1 for a, b in zip(gs, gs[1:]) if a != b) >= 100
    assert np.array_equal(s_gpu, s_ref)
    for i, (a, b) in enumerate(zip(r_gpu, r_ref)):
        assert_obs_equal(a, b, ("record", i))


def test_configuration_2_through_the_wavefront():
    """Configuration 2's lattice (1024 x 1024, random init seed 2, ambient,
    recorded every 10 steps) takes the wavefront sweep by default: 1024 tiles
    per step on every co-resident block, up to 16 steps in flight.  60 steps
    in two calls give the oracle's whole lattice, counts and records."""
    from paper_2505_05919_gb300 import workloads
    c = workloads.c2()
    K = 60
    op = oracle.physical_params(c["T"], c["P"], L=c["L"], q=c["q"], seed=c["seed"])
    with Lattice(params_from_dict(asdict(op))) as lat:
        assert lat.tiles()[0] == 6
        lat.sweep(25, c["record_every"])
        lat.sweep(K - 25, c["record_every"])
        s_gpu, o_gpu = lat.state(), lat.observables()
        r_gpu, overflow = lat.drain()
    s_ref, o_ref, r_ref = oracle_run(op, K, record_every=c["record_every"])
    assert not overflow and len(r_gpu) == len(r_ref) == K // c["record_every"]
    assert np.array_equal(s_gpu, s_ref)
    assert_obs_equal(o_gpu, o_ref)
    for i, (a, b) in enumerate(zip(r_gpu, r_ref)):
        assert_obs_equal(a, b, ("record", i))


@pytest.mark.parametrize("L,config", [(2048, 5), (2560, 4)])
def test_wavefront_sampled_windows(L, config):
    """The largest lattices the wavefront sweep takes by default (2048^2 on
    32 x 32-word tiles, 2560^2 on 64 x 64), 30 steps; windows recomputed by
    the oracle with a frozen border 2K + 2 cells wide, four across the
    periodic edges, as for the benchmark's lattices."""
    K = 30
    op = oracle.physical_params(300.0, 0.1, L=L, seed=77 + L)
    with Lattice(params_from_dict(asdict(op))) as lat:
        assert lat.tiles()[0] == config
        lat.sweep(K)
        s_gpu = lat.state()
        o_gpu = lat.observables()
        hb, co = lat.recount()
    assert (hb, co) == (o_gpu["n_hb_raw"], o_gpu["n_coop"])
    ref0 = oracle.Oracle(op)
    done, V, g, acc = oracle.volume_chain(op, ref0.observables()["V_iso"], 0, K)
    assert done == K
    assert V[-1] == pytest.approx(o_gpu["V_iso"], rel=FP_REL)
    assert o_gpu["acc_volume"] == acc
    margin, inner = 2 * K + 2, 40
    W = inner + 2 * margin
    rng = np.random.default_rng(L)
    spots = [(L - W // 2, L - W // 2), (L - W // 2, 0), (0, L - W // 2), (L - 20, L - W + 7)]
    spots += [(int(rng.integers(0, L)), int(rng.integers(0, L))) for _ in range(4)]
    full = ref0.state()
    for x0, y0 in spots:
        out = oracle.window_run(op, full, x0, y0, W, W, 0, g).reshape(L, L)
        ys = [(y0 + margin + i) % L for i in range(inner)]
        xs = [(x0 + margin + i) % L for i in range(inner)]
        assert np.array_equal(s_gpu[np.ix_(ys, xs)], out[np.ix_(ys, xs)]), (L, x0, y0)


def test_window_reads_match_the_whole_state():
    op = oracle.physical_params(300.0, 0.1, L=96, seed=12)
    with Lattice(params_from_dict(asdict(op))) as lat:
        lat.sweep(5)
        full = lat.state()
        for x0, y0, W, H in ((0, 0, 96, 96), (0, 0, 1, 1), (95, 95, 1, 1), (7, 60, 33, 36),
                             (50, 0, 46, 3)):
            assert np.array_equal(lat.window(x0, y0, W, H), full[y0:y0 + H, x0:x0 + W])
        for bad in ((-1, 0, 4, 4), (0, 0, 0, 4), (93, 0, 4, 4), (0, 95, 4, 2)):
            with pytest.raises(_capi.CvfError):
                lat.window(*bad)


@pytest.mark.parametrize("L", [65528, 65534])
def test_maximum_size_sampled_windows(L):
    """The largest lattices the library accepts (L = 65534, and 65528, the
    largest multiple of 8, which stages its tiles by TMA): cell indices up to
    4.29e9, just under 2^32.  After K steps, windows anywhere in the lattice
    (both ends of the index range included) equal the oracle's run of the
    same windows started from the init rule; V_iso follows the oracle's
    volume chain; the kept counts equal a recount."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < 2 * 2 * L * L + (4 << 30):
        pytest.skip("needs %.1f GB of free device memory" % (4 * L * L / 1e9 + 4))
    K = 3
    op = oracle.physical_params(300.0, 0.1, L=L, q=6, seed=21)
    with Lattice(params_from_dict(asdict(op))) as lat:
        lat.sweep(K)
        o = lat.observables()
        assert lat.recount() == (o["n_hb_raw"], o["n_coop"])
        done, V, g, acc = oracle.volume_chain(op, float(L * L) * op.v_iso_init, 0, K)
        assert done == K
        assert abs(o["V_iso"] - V[-1]) <= FP_REL * V[-1] and o["acc_volume"] == acc
        assert 0 < o["n_hb_raw"] <= 2 * L * L and 0 < o["n_coop"] <= 6 * L * L
        margin, inner = 2 * K + 2, 32
        W = inner + 2 * margin
        lazy = np.zeros((L, L), np.uint16)  # only the windows' pages are ever touched
        rng = np.random.default_rng(L)
        corners = [(0, 0), (L - W, 0), (0, L - W), (L - W, L - W)]
        spots = corners + [(int(rng.integers(0, L - W)), int(rng.integers(0, L - W)))
                           for _ in range(4)]
        for x0, y0 in spots:
            oracle.window_init_run(op, lazy, x0, y0, W, W, 0, g)
            want = lazy[y0 + margin:y0 + margin + inner, x0 + margin:x0 + margin + inner]
            got = lat.window(x0 + margin, y0 + margin, inner, inner)
            assert np.array_equal(got, want), (x0, y0)
