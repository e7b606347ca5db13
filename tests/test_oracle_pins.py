"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, the paper's printed indexing examples, exact enumeration
of the Boltzmann distribution of Eq. H, closed forms (binomial, truncated
Gamma, incomplete-Gamma integrals), brute-force lattice sums and exact
invariants.  No GPU is used.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from oracle import OracleParams, Oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers --
def _batch_mean(x, nbatch=50):
    """Mean and standard error from batch means (handles autocorrelation)."""
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // nbatch * nbatch
    b = x[:n].reshape(nbatch, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nbatch)


def _arms_2x2_q2(i):
    """Configurations of a 2x2 lattice with q = 2 from 16-bit integers:
    bit 4c + a is sigma of arm a of cell c.  Returns uint16 words [n, 4]."""
    i = np.asarray(i, dtype=np.int64)
    w = np.zeros((i.size, 4), np.uint16)
    for c in range(4):
        for a in range(4):
            w[:, c] |= (((i >> (4 * c + a)) & 1) << (4 * a)).astype(np.uint16)
    return w


def _counts_bruteforce(words, L):
    """N_HB_raw and N_sigma of Eq. H written out from the definitions: a bond
    joins the +x arm (0) of a cell with the -x arm (1) of its +x neighbour,
    and the +y arm (2) with the -y arm (3) of its +y neighbour (the arm
    convention of the paper's worked layout example); N_sigma counts equal
    pairs of arms inside each cell."""
    words = np.asarray(words).reshape(-1, L, L).astype(np.int64)
    arm = [(words >> (4 * a)) & 7 for a in range(4)]
    hb = (arm[0] == np.roll(arm[1], -1, axis=2)).sum(axis=(1, 2))
    hb += (arm[2] == np.roll(arm[3], -1, axis=1)).sum(axis=(1, 2))
    co = np.zeros(words.shape[0], np.int64)
    for a in range(4):
        for b in range(a + 1, 4):
            co += (arm[a] == arm[b]).sum(axis=(1, 2))
    return hb, co


def _lj_bruteforce(v, epsilon=1.0, cutoff=6.0, box=12):
    """Per-cell LJ energy summed pair by pair over every lattice vector of a
    large box: distance r |d| with r = sqrt(v) (2D monolayer of thickness r0),
    4 eps [(1/dist)^12 - (1/dist)^6] for dist < cutoff, half per cell."""
    total = 0.0
    r = math.sqrt(v)
    for i in range(-box, box + 1):
        for j in range(-box, box + 1):
            if i == 0 and j == 0:
                continue
            dist = r * math.hypot(i, j)
            if dist < cutoff:
                total += 4.0 * epsilon * (dist ** -12 - dist ** -6)
    return 0.5 * total


# ------------------------------------------------------------------ Philox --
def test_philox_known_answer_vectors():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_philox_byte_uniformity():
    rng_out = np.array([oracle.philox([c, 7, 0, 0], [123, 456]) for c in range(20000)],
                       dtype=np.uint32)
    b = rng_out.view(np.uint8).ravel()
    hist = np.bincount(b, minlength=256)
    expect = b.size / 256
    chi2 = ((hist - expect) ** 2 / expect).sum()
    # 255 degrees of freedom: mean 255, sd ~22.6; accept within ~6 sd
    assert 120 < chi2 < 400


# ---------------------------------------------------------- paper examples --
def test_paper_layout_example():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_layout_example.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 17
    for r in rows:
        N, L, cell, arm, idx = map(int, r[:5])
        c2, a2 = oracle.bond_partner(L, cell, arm)
        assert a2 * N + c2 == idx
        # the relation is symmetric: the partner's partner is the cell itself
        assert oracle.bond_partner(L, c2, a2) == (cell, arm)


def test_physical_units_table1():
    # kT/eps and P v0/eps for eps = 5.5 kJ/mol and r0 = 2.9 A (Table 1)
    assert oracle.physical_params(300, 0.1).kT == pytest.approx(0.453516, abs=2e-6)
    assert oracle.physical_params(270, 0.1).kT == pytest.approx(0.408165, abs=2e-6)
    assert oracle.physical_params(330, 0.1).kT == pytest.approx(0.498868, abs=2e-6)
    assert oracle.physical_params(300, 0.1).P == pytest.approx(2.6704e-4, rel=1e-4)
    assert oracle.physical_params(300, 50).P == pytest.approx(0.133522, rel=1e-5)


# -------------------------------------------------------- LJ lattice sums --
@pytest.mark.parametrize("v", [1.0, 1.1, 2 ** (1 / 3), 1.5, 2.0, 2.5, 36 / 26 - 1e-9, 36 / 26 + 1e-9, 7.0])
def test_lj_cell_energy_matches_pairwise_sum(v):
    got = oracle.lj_cell_energy(v, 1.0, 6.0)
    want = _lj_bruteforce(v)
    assert got == pytest.approx(want, rel=1e-12, abs=1e-15)
    assert oracle.lj_cell_energy(v, 0.0, 6.0) == 0.0


def test_shell_multiplicities():
    d2, m = oracle.shell_table(6.0)
    # every lattice vector with |d|^2 < 36 exactly once
    n_vec = sum(1 for i in range(-6, 7) for j in range(-6, 7) if 0 < i * i + j * j < 36)
    assert m.sum() == n_vec
    assert list(d2[:6]) == [1, 2, 4, 5, 8, 9] and list(m[:6]) == [4, 4, 4, 8, 4, 4]


# --------------------------------------------- single-variable detailed balance --
def _detailed_balance_check(p, cfgs, g, rev_cfgs=None):
    """For every configuration, cell, arm and proposal offset k, the oracle's
    move sigma -> sigma' is accepted with probability T/2^32; check
    pi(sigma) A(sigma->sigma') = pi(sigma') A(sigma'->sigma) with pi from
    Eq. H at fixed volume, to the 2^-32 resolution of the thresholds."""
    L, q = p.L, p.q
    N = L * L
    s_new, T = oracle.arm_probe_all(p, cfgs, g)
    J_eff = p.J - p.P * p.v_HB
    hb, co = _counts_bruteforce(cfgs, L)
    E = -(g * J_eff) * hb - p.J_sigma * co
    n = cfgs.shape[0]
    worst = 0.0
    for c in range(N):
        for a in range(4):
            for k in range(q - 1):
                new = cfgs.copy()
                sp = s_new[:, c, a, k].astype(np.uint16)
                s_old = (cfgs[:, c] >> (4 * a)) & 7
                assert np.all(sp != s_old) and np.all(sp < q)
                assert np.all(sp == (s_old + 1 + k) % q)
                new[:, c] = (new[:, c] & ~np.uint16(7 << (4 * a))) | (sp << (4 * a))
                hb2, co2 = _counts_bruteforce(new, L)
                E2 = -(g * J_eff) * hb2 - p.J_sigma * co2
                dE = E2 - E
                # reverse proposal offset from sigma' back to sigma
                krev = (s_old.astype(np.int64) - sp.astype(np.int64) - 1) % q
                s_back, T_back = oracle.arm_probe_all(p, new, g)
                tb = T_back[np.arange(n), c, a, krev]
                assert np.all(s_back[np.arange(n), c, a, krev] == s_old)
                fwd = T[:, c, a, k].astype(np.float64) / 2 ** 32
                bwd = tb.astype(np.float64) / 2 ** 32
                lhs = fwd
                rhs = bwd * np.exp(-dE / p.kT)
                # A = min(1, exp(-dE/kT)) to within 2^-32 absolute
                err = np.abs(lhs - rhs) / np.maximum(np.maximum(lhs, rhs), 1e-300)
                bound = 2.0 ** -32 / np.maximum(np.minimum(fwd, bwd), 2.0 ** -32) + 1e-12
                assert np.all(err <= bound)
                worst = max(worst, float(err.max()))
    return worst


@pytest.mark.parametrize("g", [0, 1])
def test_detailed_balance_2x2_q2_all_states(g):
    p = OracleParams(L=2, q=2, kT=0.9, P=0.3, J=2.0, J_sigma=0.32, v_HB=0.6)
    cfgs = _arms_2x2_q2(np.arange(1 << 16))
    _detailed_balance_check(p, cfgs, g)


def test_detailed_balance_4x4_q3_sampled():
    rng = np.random.default_rng(11)
    p = OracleParams(L=4, q=3, kT=0.7, P=0.05)
    arms = rng.integers(0, 3, size=(60, 16, 4))
    cfgs = np.zeros((60, 16), np.uint16)
    for a in range(4):
        cfgs |= (arms[:, :, a] << (4 * a)).astype(np.uint16)
    _detailed_balance_check(p, cfgs, 1)


# ------------------------------------------------ exact enumeration averages --
def _exact_2x2_q2(p, g=1):
    cfgs = _arms_2x2_q2(np.arange(1 << 16))
    hb, co = _counts_bruteforce(cfgs, 2)
    J_eff = p.J - p.P * p.v_HB
    E = -(g * J_eff) * hb - p.J_sigma * co
    wgt = np.exp(-(E - E.min()) / p.kT)
    Z = wgt.sum()
    return (wgt * hb).sum() / Z, (wgt * co).sum() / Z


@pytest.mark.parametrize("kT", [0.8, 1.6])
@pytest.mark.parametrize("schedule", [oracle.SCHED_CHECKERBOARD, oracle.SCHED_LAYERED])
@pytest.mark.parametrize("rng_words", [1, 2])
def test_enumeration_averages_2x2_q2(kT, schedule, rng_words):
    p = OracleParams(L=2, q=2, kT=kT, P=0.1, volume_moves=0, schedule=schedule,
                     rng_words=rng_words, seed=1000 + int(kT * 10) + 7 * schedule + rng_words)
    o = Oracle(p)
    rec = o.run(60000, record_every=1)
    hb = np.array([r["n_hb_raw"] for r in rec])[2000:]
    co = np.array([r["n_coop"] for r in rec])[2000:]
    ehb, eco = _exact_2x2_q2(p)
    m, se = _batch_mean(hb)
    assert abs(m - ehb) < 5 * se + 1e-9, (m, se, ehb)
    m, se = _batch_mean(co)
    assert abs(m - eco) < 5 * se + 1e-9, (m, se, eco)


# ---------------------------------------------------------------- limits --
def test_high_temperature_limit_binomial():
    # kT -> infinity: every threshold is 2^32, every proposal is accepted and
    # the sigma stay independent and uniform, so N_HB_raw ~ Binomial(2N, 1/q)
    # and <N_sigma> = 6N/q with variance 6N (1/q)(1-1/q).
    L, q = 16, 6
    p = OracleParams(L=L, q=q, kT=1e300, volume_moves=0, seed=5)
    assert np.all(oracle.threshold_table(p) == 2 ** 32)
    o = Oracle(p)
    rec = o.run(8000, record_every=4)
    N = L * L
    hb = np.array([r["n_hb_raw"] for r in rec], dtype=np.float64)
    co = np.array([r["n_coop"] for r in rec], dtype=np.float64)
    assert rec[-1]["acc_sigma"] == 8000 * 4 * N
    m, se = _batch_mean(hb)
    assert abs(m - 2 * N / q) < 5 * se
    var_expect = 2 * N * (1 / q) * (1 - 1 / q)
    assert abs(hb.var() / var_expect - 1) < 0.15
    m, se = _batch_mean(co)
    assert abs(m - 6 * N / q) < 5 * se
    assert abs(co.var() / (6 * N / q * (1 - 1 / q)) - 1) < 0.15


@pytest.mark.parametrize("volume_moves", [0, 1])
def test_ground_state_is_frozen(volume_moves):
    # ordered init (all sigma equal: every bond formed, every pair equal),
    # liquid gate, J_eff > 0, kT -> 0: every proposal loses one bond and three
    # cooperative pairs, its threshold is 0 and it is always rejected.
    L = 8
    N = L * L
    p = OracleParams(L=L, q=6, kT=1e-3, init=oracle.INIT_ORDERED, volume_moves=volume_moves,
                     dv_max_frac=0.001)
    o = Oracle(p)
    s0 = o.state()
    o.run(40)
    assert np.array_equal(o.state(), s0)
    ob = o.observables()
    assert ob["n_hb_raw"] == 2 * N and ob["n_coop"] == 6 * N and ob["acc_sigma"] == 0
    v = ob["V_iso"] / N
    H = N * _lj_bruteforce(v) - p.J * 2 * N - p.J_sigma * 6 * N + p.P * (ob["V_iso"] + p.v_HB * 2 * N)
    assert ob["H"] == pytest.approx(H, rel=1e-12)
    assert ob["U_LJ"] == pytest.approx(N * _lj_bruteforce(v), rel=1e-12)


def test_incremental_counters_equal_recount():
    p = OracleParams(L=16, q=6, kT=0.6, seed=3)
    o = Oracle(p)
    for _ in range(60):
        o.step()
        ob = o.observables()
        hb, co = o.recount()
        hb2, co2 = _counts_bruteforce(o.state().ravel(), 16)
        assert (ob["n_hb_raw"], ob["n_coop"]) == (hb, co) == (int(hb2[0]), int(co2[0]))
        assert 0 <= hb <= 2 * 256 and 0 <= co <= 6 * 256


def test_checkpoint_resume_bit_exact():
    p = OracleParams(L=16, q=6, kT=0.5, seed=9, dv_max_frac=0.05)
    a = Oracle(p)
    a.run(62)
    b = Oracle(p)
    b.run(37)
    ob = b.observables()
    c = Oracle(p, state=b.state(), V_iso=ob["V_iso"], sweep=ob["sweep"])
    c.run(25)
    oa, oc = a.observables(), c.observables()
    assert np.array_equal(a.state(), c.state())
    for k in ("sweep", "n_hb_raw", "n_coop", "V_iso", "H", "g"):
        assert oa[k] == oc[k]


def test_layer_order_is_uniform_permutation():
    p = OracleParams(seed=21)
    counts = {}
    for s in range(24000):
        o = tuple(oracle.layer_order(p, s))
        assert sorted(o) == [0, 1, 2, 3]
        counts[o] = counts.get(o, 0) + 1
    assert len(counts) == 24
    c = np.array(list(counts.values()), dtype=np.float64)
    chi2 = ((c - 1000) ** 2 / 1000).sum()
    assert chi2 < 60  # 23 degrees of freedom


# ------------------------------------------------------------ volume move --
def test_volume_move_truncated_gamma():
    # With J = J_sigma = v_HB = 0 and no LJ term the isobaric weight of V_iso
    # is V^N exp(-P V / kT) on V >= N v0 (hard core): a truncated Gamma whose
    # mean is (N+1) Q(N+2, bN) / (b Q(N+1, bN)), b = P/kT.
    L = 4
    N = L * L
    for P, seed in ((0.5, 1), (2.0, 2)):
        p = OracleParams(L=L, q=6, epsilon=0.0, J=0.0, J_sigma=0.0, v_HB=0.0, kT=1.0, P=P,
                         v_iso_init=1.5, dv_max_frac=0.25, seed=seed)
        o = Oracle(p)
        rec = o.run(300000, record_every=5)
        V = np.array([r["V_iso"] for r in rec])[1000:]
        b = P / p.kT
        mean = (N + 1) * special.gammaincc(N + 2, b * N) / (b * special.gammaincc(N + 1, b * N))
        m, se = _batch_mean(V, 100)
        assert abs(m - mean) < 5 * se, (P, m, se, mean)
        assert V.min() >= N


def test_volume_move_gate_joint_distribution():
    # 2x2 lattice, q = 2, LJ off: the joint weight of (sigma, V_iso) is
    # V^N exp(-[P V - g(V) J_eff N_HB_raw - J_sigma N_sigma]/kT) with the gate
    # g(V) = [V < 2 N v0] (Eq. H with theta(r_1/2 - r)).  Integrate V out
    # exactly with incomplete Gamma functions and compare <N_HB_raw>, <V_iso>
    # and the liquid fraction with a long run.
    N = 4
    kT, P = 3.0, 0.9
    p = OracleParams(L=2, q=2, epsilon=0.0, kT=kT, P=P, v_iso_init=1.5, dv_max_frac=0.4, seed=77)
    cfgs = _arms_2x2_q2(np.arange(1 << 16))
    hb, co = _counts_bruteforce(cfgs, 2)
    b = P / kT
    J_eff = p.J - p.P * p.v_HB

    def I(k, lo, hi):  # int_lo^hi V^k e^{-bV} dV
        g = math.gamma(k + 1) / b ** (k + 1)
        up = special.gammaincc(k + 1, b * lo) - (special.gammaincc(k + 1, b * hi) if hi != math.inf else 0.0)
        return g * up

    I0l, I0g = I(N, N, 2 * N), I(N, 2 * N, math.inf)
    I1l, I1g = I(N + 1, N, 2 * N), I(N + 1, 2 * N, math.inf)
    wl = np.exp((J_eff * hb + p.J_sigma * co) / kT)
    wg = np.exp(p.J_sigma * co / kT)
    Z = (wl * I0l + wg * I0g).sum()
    e_hb = ((wl * I0l + wg * I0g) * hb).sum() / Z
    e_V = (wl * I1l + wg * I1g).sum() / Z
    e_liq = (wl * I0l).sum() / Z
    o = Oracle(p)
    rec = o.run(400000, record_every=2)[2000:]
    hbs = np.array([r["n_hb_raw"] for r in rec], dtype=np.float64)
    Vs = np.array([r["V_iso"] for r in rec])
    liq = np.array([r["g"] for r in rec], dtype=np.float64)
    for arr, want in ((hbs, e_hb), (Vs, e_V), (liq, e_liq)):
        m, se = _batch_mean(arr, 100)
        assert abs(m - want) < 5 * se, (m, se, want)
    assert 0.2 < e_liq < 0.8  # both phases sampled


def test_volume_move_lj_marginal():
    # J = J_sigma = v_HB = 0 with the LJ term on: the V_iso marginal is
    # V^N exp(-[N u(V/N) + P V]/kT) on V >= N, with u the pairwise lattice sum.
    L = 4
    N = L * L
    kT, P = 1.0, 1.0
    p = OracleParams(L=L, q=6, J=0.0, J_sigma=0.0, v_HB=0.0, kT=kT, P=P, dv_max_frac=0.03,
                     v_iso_init=1.3, seed=31)
    vs = np.linspace(1.0, 4.0, 6001)
    logw = np.array([N * math.log(N * v) - (N * _lj_bruteforce(v, box=8) + P * N * v) / kT for v in vs])
    w = np.exp(logw - logw.max())
    mean_v = integrate.trapezoid(w * vs, vs) / integrate.trapezoid(w, vs)
    o = Oracle(p)
    rec = o.run(200000, record_every=5)[1000:]
    v = np.array([r["V_iso"] for r in rec]) / N
    m, se = _batch_mean(v, 100)
    assert abs(m - mean_v) < 5 * se + 2e-4, (m, se, mean_v)


@pytest.mark.parametrize("init", [oracle.INIT_RANDOM, oracle.INIT_ORDERED])
def test_window_init_run_matches_whole_lattice(init):
    """A window started by the init rule alone (the rest of the lattice left
    zero) and run K steps agrees with the whole lattice more than 2K + 2
    cells inside its border: the tool behind the sampled checks of lattices
    too large for the oracle to hold."""
    L, K = 40, 3
    op = oracle.physical_params(300.0, 0.1, L=L, seed=17, init=init)
    ref = oracle.Oracle(op)
    start = ref.state().copy()
    done, V, g, _ = oracle.volume_chain(op, ref.observables()["V_iso"], 0, K)
    assert done == K
    ref.run(K)
    whole = np.zeros((L, L), np.uint16)
    oracle.window_init_run(op, whole, 0, 0, L, L, 0, [])
    assert np.array_equal(whole, start)          # the init rule, cell by cell
    w = np.zeros((L, L), np.uint16)
    x0, y0, W, H = 3, 5, 30, 32
    oracle.window_init_run(op, w, x0, y0, W, H, 0, g)
    m = 2 * K + 2
    inner = (slice(y0 + m, y0 + H - m), slice(x0 + m, x0 + W - m))
    assert np.array_equal(w[inner], ref.state()[inner])
    assert not w[:y0].any() and not w[:, :x0].any()  # nothing written outside


@pytest.mark.parametrize("init,dv,T", [(oracle.INIT_RANDOM, 0.01, 300.0),
                                       (oracle.INIT_ORDERED, 0.05, 330.0),
                                       (oracle.INIT_RANDOM, 0.4, 900.0)])
def test_volume_chain_equals_full_run(init, dv, T):
    """The V_iso chain run alone (orc_volume_chain, the V reference of the
    sampled checks at large sizes) reproduces the V_iso and gate of every
    step of the full MC run up to its first gate-changing proposal, and its
    acceptance count equals the run's over the steps it covers; with large
    moves from v = 1.9 the chain must stop early, exactly where the full run
    meets the first proposal that would change the gate."""
    L, K = 6, 400
    op = oracle.physical_params(T, 0.1, L=L, seed=23, init=init, dv_max_frac=dv,
                                v_iso_init=1.9 if dv > 0.1 else 2 ** (1 / 3))
    ref = Oracle(op)
    V0 = ref.observables()["V_iso"]
    done, V, g, acc = oracle.volume_chain(op, V0, 0, K)
    rec = ref.run(K, record_every=1)
    assert len(rec) == K
    Vr = np.array([r["V_iso"] for r in rec])
    gr = np.array([r["g"] for r in rec])
    accr = np.array([r["acc_volume"] for r in rec])
    assert np.array_equal(V[:done], Vr[:done])
    assert np.array_equal(g[:done], gr[:done])
    if done == K:
        assert acc == accr[-1]
    else:
        # step `done` proposes a gate change: recompute that proposal here
        # from the Philox words (tag 3, cell word 2^32 - 1) and the rule
        # dV = (2 u1 - 1) dV_max of the volume move
        r = oracle.philox([0xFFFFFFFF, done & 0xFFFFFFFF, done >> 32, 3],
                          [op.seed & 0xFFFFFFFF, op.seed >> 32])
        u1 = ((int(r[0]) << 21) | (int(r[1]) >> 11)) / 2.0 ** 53
        N = L * L
        dV = (2.0 * u1 - 1.0) * (dv * N * op.v_iso_init)
        v_before = (Vr[done - 1] if done > 0 else V0) / N
        v_new = v_before + dV / N
        assert v_new >= 1.0 and (v_new < 2.0) != (v_before < 2.0)
    if dv > 0.1:
        assert done < K  # this case must exercise the early stop


def test_volume_chain3_equals_full_run():
    """The 3D V_iso chain with the bond count held fixed equals the full
    cubic run's V_iso at every step while the gate cannot change."""
    L, K = 4, 300
    op = oracle.physical_params3(300.0, 0.1, L=L, seed=29)
    ref = oracle.Oracle3(op)
    ob = ref.observables()
    V, acc = oracle.volume_chain3(op, ob["V_iso"], ob["n_hb_raw"], 0, K)
    rec = ref.run(K, record_every=1)
    Vr = np.array([r["V_iso"] for r in rec])
    assert all(r["g"] == 1 for r in rec)
    assert np.array_equal(V, Vr)
    assert acc == rec[-1]["acc_volume"]


def test_window_across_the_periodic_edges_matches_whole_lattice():
    """A window that runs across both periodic edges (cells taken mod L)
    agrees with the whole lattice more than 2K + 2 cells inside, like one
    that lies inside the lattice."""
    L, K = 40, 3
    op = oracle.physical_params(300.0, 0.1, L=L, seed=29)
    ref = oracle.Oracle(op)
    done, V, g, _ = oracle.volume_chain(op, ref.observables()["V_iso"], 0, K)
    assert done == K
    ref.run(K)
    w = np.zeros((L, L), np.uint16)
    x0, y0, W, H = 30, 33, 24, 22   # x 30..53 -> 30..39, 0..13; y 33..54 -> 33..39, 0..14
    oracle.window_init_run(op, w, x0, y0, W, H, 0, g)
    m = 2 * K + 2
    ys = [(y0 + i) % L for i in range(m, H - m)]
    xs = [(x0 + i) % L for i in range(m, W - m)]
    assert np.array_equal(w[np.ix_(ys, xs)], ref.state()[np.ix_(ys, xs)])
    # nothing outside the window was written
    inside = np.zeros((L, L), bool)
    inside[np.ix_([(y0 + i) % L for i in range(H)], [(x0 + i) % L for i in range(W)])] = True
    assert not w[~inside].any()
