"""GPU parity of the cubic-lattice path (``cvf3_*``) against the 3D oracle.

Same seeded inputs on both sides; the packed lattice, every integer counter
and N_q' must be bit-identical, FP64 observables within rel 1e-12 (both sides
evaluate the same IEEE operations in the same order, so they are in practice
equal).  Sizes cover the 16-byte-vector path (L % 4 == 0) and the per-cell
path (odd L, L = 2 with a neighbour on both sides, N % 4 != 0 tails), the
graph-captured steps and the steps launched one by one, both inits, three
(T, P) points, gate flips of the volume move, the 64-bit threshold compare,
checkpoint/resume, and the paper's largest cube (260^3 = 17 576 000 cells).
"""
from dataclasses import asdict

import numpy as np
import pytest

import oracle
from paper_2505_05919_gb300 import Lattice3, _capi, params_from_dict

pytestmark = pytest.mark.gpu

INT_KEYS = ("sweep", "n_hb", "n_hb_raw", "n_coop", "acc_sigma", "acc_volume", "g")
FP_KEYS = ("V_iso", "V", "U_LJ", "H")
REL = 1e-12


def _same(got, want, ctx=""):
    for k in INT_KEYS:
        assert got[k] == want[k], (ctx, k, got[k], want[k])
    assert list(got["n_state"]) == list(want["n_state"]), ctx
    for k in FP_KEYS:
        assert abs(got[k] - want[k]) <= REL * abs(want[k]), (ctx, k, got[k], want[k])


def _run_both(op, steps, record_every=0):
    """The cube run on the GPU and by the oracle: (state, observables,
    recount, series, eta configurations) of each."""
    ref = oracle.Oracle3(op)
    want_series = ref.run(steps, record_every)
    with Lattice3(params_from_dict(asdict(op))) as lat:
        lat.sweep(steps, record_every)
        got_series, overflow = lat.drain()
        assert not overflow
        return (lat.state(), lat.observables(), lat.recount(), got_series, lat.eta()), \
               (ref.state(), ref.observables(), ref.recount(), want_series, ref.eta())


# (L, eta moves): odd sides run with eta = 1 (the cube partition needs an even L)
SIDES = [(2, 1), (3, 0), (4, 1), (4, 0), (5, 0), (6, 1), (8, 1), (12, 1), (16, 1), (16, 0)]


@pytest.mark.parametrize("L,eta", SIDES)
@pytest.mark.parametrize("init", [oracle.INIT_RANDOM, oracle.INIT_ORDERED])
def test_lattice3_matches_oracle(L, eta, init):
    op = oracle.physical_params3(300.0, 0.1, L=L, init=init, seed=100 + L, eta_moves=eta)
    got, want = _run_both(op, 45)
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[4], want[4])   # the cube configurations (eta)
    _same(got[1], want[1], (L, init))
    assert got[2] == want[2] == (want[1]["n_hb_raw"], want[1]["n_coop"])


@pytest.mark.parametrize("T,P", [(270.0, 0.1), (300.0, 25.0), (330.0, 50.0)])
@pytest.mark.parametrize("q", [3, 6, 8])
def test_lattice3_state_points(T, P, q):
    op = oracle.physical_params3(T, P, L=8, q=q, seed=int(T) + q, dv_max_frac=0.05)
    got, want = _run_both(op, 40)
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[4], want[4])
    _same(got[1], want[1], (T, P, q))


@pytest.mark.parametrize("L,every", [(5, 3), (8, 1), (12, 7)])
def test_lattice3_series_matches_oracle(L, every):
    op = oracle.physical_params3(285.0, 10.0, L=L, seed=7 + L, dv_max_frac=0.05,
                                 eta_moves=1 - L % 2)
    got, want = _run_both(op, 70, record_every=every)
    assert len(got[3]) == len(want[3]) == 70 // every
    for i, (g, w) in enumerate(zip(got[3], want[3])):
        _same(g, w, ("record", i))


@pytest.mark.parametrize("L,P,kT", [(2, 1.2, 3.0), (3, 2.0, 5.0), (4, 3.0, 5.0)])
def test_lattice3_gate_flips(L, P, kT):
    # small hot cubes near v = 2 whose volume moves cross the liquid/gas gate,
    # so the move of the next step is sometimes decided only after the bonds
    op = oracle.params3(L=L, kT=kT, P=P, epsilon=0.0, v_iso_init=1.9, dv_max_frac=0.2, seed=31,
                        eta_moves=1 - L % 2)
    got, want = _run_both(op, 300, record_every=1)
    gates = [r["g"] for r in want[3]]
    assert sum(a != b for a, b in zip(gates, gates[1:])) >= 3
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[4], want[4])
    for i, (g, w) in enumerate(zip(got[3], want[3])):
        _same(g, w, ("record", i))


def test_lattice3_cmp64_ground_state():
    # kT -> 0: thresholds of 0 (the 64-bit compare) and a frozen ordered cube
    op = oracle.params3(L=8, kT=1e-3, init=oracle.INIT_ORDERED, dv_max_frac=0.001, seed=3)
    assert (oracle.threshold_table3(op) == 0).any()
    got, want = _run_both(op, 40)
    assert not got[0].any() and np.array_equal(got[0], want[0])
    assert np.array_equal(got[4], want[4])
    _same(got[1], want[1])
    # every allowed edge bonded: 2N of them with eta (3N without)
    assert got[1]["n_hb_raw"] == 2 * 512 and got[1]["n_coop"] == 15 * 512


def test_lattice3_checkpoint_resume():
    op = oracle.physical_params3(300.0, 0.1, L=12, seed=41, dv_max_frac=0.05)
    mid = oracle.Oracle3(op)
    mid.run(17)
    ob = mid.observables()
    ref = oracle.Oracle3(op)
    ref.run(50)
    with Lattice3(params_from_dict(asdict(op))) as lat:
        lat.sweep(3)                     # overwritten by set_state and set_eta
        lat.set_state(mid.state(), ob["V_iso"], ob["sweep"])
        lat.set_eta(mid.eta())
        assert np.array_equal(lat.eta(), mid.eta())
        assert lat.observables()["n_hb_raw"] == ob["n_hb_raw"]
        lat.sweep(33)
        s, o, e = lat.state(), lat.observables(), lat.eta()
    assert np.array_equal(s, ref.state())
    assert np.array_equal(e, ref.eta())
    want = ref.observables()
    for k in ("sweep", "n_hb_raw", "n_coop", "g", "n_state"):
        assert o[k] == want[k], k
    for k in FP_KEYS:
        assert abs(o[k] - want[k]) <= REL * abs(want[k]), k


def test_lattice3_calls_split_like_one_run():
    op = oracle.physical_params3(300.0, 0.1, L=6, seed=5)
    ref = oracle.Oracle3(op)
    ref.run(80)
    with Lattice3(params_from_dict(asdict(op))) as lat:
        for n in (0, 1, 31, 32, 5, 11):
            lat.sweep(n)
        assert np.array_equal(lat.state(), ref.state())
        _same(lat.observables(), ref.observables())


def test_lattice3_rejects_bad_eta():
    op = oracle.physical_params3(300.0, 0.1, L=4, q=6)
    with Lattice3(params_from_dict(asdict(op))) as lat:
        cfg = lat.eta()
        assert cfg.size == 16 and cfg.max() <= 8
        bad = cfg.copy()
        bad[3] = 9
        with pytest.raises(_capi.CvfError):
            lat.set_eta(bad)
        with pytest.raises(_capi.CvfError):
            lat.set_eta(cfg[:-1])
        assert np.array_equal(lat.eta(), cfg)
    with Lattice3(params_from_dict(asdict(oracle.physical_params3(300.0, 0.1, L=4, eta_moves=0)))) as lat:
        with pytest.raises(_capi.CvfError):
            lat.set_eta(np.zeros(16, np.uint8))
    with pytest.raises(_capi.CvfError):  # eta moves need an even side
        Lattice3(params_from_dict(asdict(oracle.physical_params3(300.0, 0.1, L=5, eta_moves=0))
                                  | {"eta_moves": 1}))


def test_lattice3_rejects_bad_state():
    op = oracle.physical_params3(300.0, 0.1, L=4, q=6)
    with Lattice3(params_from_dict(asdict(op))) as lat:
        good = lat.state()
        for bad_word in (6, 6 << 20, 1 << 24, 1 << 3, 1 << 23):
            w = good.copy().reshape(-1)
            w[5] = bad_word
            with pytest.raises(_capi.CvfError):
                lat.set_state(w, 64 * 1.5)
        with pytest.raises(_capi.CvfError):
            lat.set_state(good, 63.0)     # V_iso below the hard core N v0
        assert np.array_equal(lat.state(), good)


@pytest.mark.parametrize("L,steps", [(130, 3), (128, 4), (260, 2)])
def test_lattice3_large_cubes(L, steps):
    # full-size parity: the largest cube of the paper's scaling runs (260^3)
    # and a large cube on the per-cell path (130^3), whole lattice compared
    op = oracle.physical_params3(300.0, 0.1, L=L, seed=3)
    got, want = _run_both(op, steps)
    assert np.array_equal(got[0], want[0])
    assert np.array_equal(got[4], want[4])
    _same(got[1], want[1], L)


@pytest.mark.parametrize("L,steps,extra", [
    (16, 120, {}),
    (24, 60, dict(q=8, init=oracle.INIT_ORDERED)),
    (32, 40, dict(T=330.0, P=50.0)),
    (64, 12, {}),
    (16, 100, dict(kT=1e-3, init=oracle.INIT_ORDERED)),                 # 64-bit compare
    # gate flips: no bond or LJ bias, v fluctuating about the gate at v = 2
    (16, 200, dict(kT=1.0, P=0.5, J=0.0, v_HB=0.0, epsilon=0.0, v_iso_init=1.98, dv_max_frac=0.02)),
])
@pytest.mark.parametrize("eta_moves", [1, 0])
def test_lattice3_resident_cluster(L, steps, extra, eta_moves):
    """The cube resident in one thread-block cluster for each call gives the
    oracle's lattice, cube configurations, counts, N_q' and recorded series
    -- with the eta step (the cubes whose lower plane lies in a CTA's slab
    move there, their upper corners possibly in the next CTA's shared
    memory) and without it (eta = 1)."""
    extra = dict(extra, eta_moves=eta_moves)
    if "kT" in extra:
        op = oracle.params3(L=L, seed=500 + L, **extra)
    else:
        T, P = extra.pop("T", 300.0), extra.pop("P", 0.1)
        op = oracle.physical_params3(T, P, L=L, seed=500 + L, dv_max_frac=0.05, **extra)
    ref = oracle.Oracle3(op)
    want = ref.run(steps, 1)
    if extra.get("dv_max_frac") == 0.02:
        gates = [r["g"] for r in want]
        assert sum(a != b for a, b in zip(gates, gates[1:])) >= 10
    with Lattice3(params_from_dict(asdict(op))) as lat:
        lat.set_resident(1)
        assert lat.resident()
        lat.sweep(steps // 3, 1)
        lat.sweep(steps - steps // 3, 1)   # two calls: the cube leaves and re-enters the cluster
        s, o = lat.state(), lat.observables()
        eta = lat.eta() if eta_moves else None
        got, overflow = lat.drain()
        assert lat.recount() == (o["n_hb_raw"], o["n_coop"])
    assert not overflow and len(got) == len(want) == steps
    assert np.array_equal(s, ref.state())
    if eta_moves:
        assert np.array_equal(eta, ref.eta())
    _same(o, ref.observables(), L)
    for i, (g, w) in enumerate(zip(got, want)):
        _same(g, w, ("record", i))


def test_lattice3_resident_choice():
    with Lattice3(params_from_dict(asdict(oracle.physical_params3(300.0, 0.1, L=16, eta_moves=0)))) as lat:
        assert lat.resident()              # small cubes run resident by default
        lat.set_resident(0)
        assert not lat.resident()
    with Lattice3(params_from_dict(asdict(oracle.physical_params3(300.0, 0.1, L=16)))) as lat:
        assert lat.resident()              # with the eta step as well
    with Lattice3(params_from_dict(asdict(oracle.physical_params3(300.0, 0.1, L=32)))) as lat:
        assert lat.resident()              # 32^3 in a 16-CTA cluster
    with Lattice3(params_from_dict(asdict(oracle.physical_params3(300.0, 0.1, L=40)))) as lat:
        assert not lat.resident()          # beyond 32^3 the launch form is faster
    with Lattice3(params_from_dict(asdict(oracle.physical_params3(300.0, 0.1, L=12)))) as lat:
        assert not lat.resident()          # 12 is not a multiple of 8
        with pytest.raises(_capi.CvfError):
            lat.set_resident(1)


def test_lattice3_window_reads_match_the_whole_state():
    op = oracle.physical_params3(300.0, 0.1, L=20, seed=8)
    with Lattice3(params_from_dict(asdict(op))) as lat:
        lat.sweep(3)
        full = lat.state()
        for x0, y0, z0, W, H, D in ((0, 0, 0, 20, 20, 20), (19, 19, 19, 1, 1, 1),
                                    (3, 5, 7, 11, 9, 13), (0, 17, 2, 20, 3, 1)):
            assert np.array_equal(lat.window(x0, y0, z0, W, H, D),
                                  full[z0:z0 + D, y0:y0 + H, x0:x0 + W])
        for bad in ((-1, 0, 0, 2, 2, 2), (0, 0, 0, 2, 0, 2), (0, 0, 19, 2, 2, 2)):
            with pytest.raises(_capi.CvfError):
                lat.window(*bad)


@pytest.mark.parametrize("L", [1024, 1021])
def test_lattice3_maximum_size_sampled_boxes(L):
    """The largest cubes the library accepts (1024^3 = 1.07e9 cells on the
    16-byte group path; 1021^3 on the per-cell path): after K steps, boxes
    at opposite corners and random places equal the oracle's run of the same
    boxes started from the init rule; V_iso follows the volume chain; the
    kept counts equal a recount."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < 4 * L ** 3 + (4 << 30):
        pytest.skip("needs %.1f GB of free device memory" % (4 * L ** 3 / 1e9 + 4))
    K = 2
    op = oracle.physical_params3(300.0, 0.1, L=L, seed=23, eta_moves=1 - L % 2)
    N = L ** 3
    with Lattice3(params_from_dict(asdict(op))) as lat:
        ob0 = lat.observables()
        lat.sweep(K)
        o = lat.observables()
        assert lat.recount() == (o["n_hb_raw"], o["n_coop"])
    V, acc = oracle.volume_chain3(op, float(N) * op.v_iso_init, ob0["n_hb_raw"], 0, K)
    gates = [int(v / N < 2.0) for v in V]
    assert all(gg == ob0["g"] for gg in gates)   # no gate change: the chain needs no bonds
    assert abs(o["V_iso"] - V[-1]) <= REL * V[-1] and o["acc_volume"] == acc
    assert 0 < o["n_hb_raw"] <= (2 if op.eta_moves else 3) * N and 0 < o["n_coop"] <= 15 * N
    # a step carries information two cells along each axis, three with eta moves
    margin, inner = (3 if op.eta_moves else 2) * K + 2, 16
    W = inner + 2 * margin
    rng = np.random.default_rng(L)
    spots = [(0, 0, 0), (L - W, L - W, L - W), (L - W, 0, L - W), (0, L - W, 0)]
    spots += [tuple(int(v) for v in rng.integers(0, L - W, 3)) for _ in range(4)]
    lazy = np.zeros(N, np.uint32)  # only the boxes' pages are ever touched
    lazy_eta = np.zeros(N // 4 if op.eta_moves else 1, np.uint8)
    cube = lazy.reshape(L, L, L)
    with Lattice3(params_from_dict(asdict(op))) as lat:
        lat.sweep(K)
        for x0, y0, z0 in spots:
            oracle.window_init_run3(op, lazy, x0, y0, z0, W, W, W, 0, gates,
                                    lazy_eta if op.eta_moves else None)
            want = cube[z0 + margin:z0 + margin + inner, y0 + margin:y0 + margin + inner,
                        x0 + margin:x0 + margin + inner]
            got = lat.window(x0 + margin, y0 + margin, z0 + margin, inner, inner, inner)
            assert np.array_equal(got, want), (x0, y0, z0)


@pytest.mark.parametrize("T,P,init", [(270.0, 0.1, oracle.INIT_RANDOM), (330.0, 50.0, oracle.INIT_RANDOM),
                                      (300.0, 0.1, oracle.INIT_ORDERED)])
def test_lattice3_eta_every_step(T, P, init):
    """The eta update of App. A on the GPU follows the oracle step by step:
    the cube configurations, the recorded counts of every step (N_HB_raw
    counts bonds on allowed edges only) and the final lattice."""
    op = oracle.physical_params3(T, P, L=8, seed=71, init=init, dv_max_frac=0.05)
    ref = oracle.Oracle3(op)
    with Lattice3(params_from_dict(asdict(op))) as lat:
        assert np.array_equal(lat.eta(), ref.eta())      # the initial configurations
        for chunk in (1, 2, 5, 40):
            want = ref.run(chunk, 1)
            lat.sweep(chunk, 1)
            got, _ = lat.drain()
            for g, w in zip(got, want):
                _same(g, w, (T, P, chunk))
            assert np.array_equal(lat.eta(), ref.eta())
        assert np.array_equal(lat.state(), ref.state())
    assert ref.acc_eta > 0
