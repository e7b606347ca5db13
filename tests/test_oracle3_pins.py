"""Pins of the 3D oracle (cubic lattice, six arms, layered schedule) against
what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
indexing examples the paper prints for its N = 64 cubic lattice (Sec. II.C,
Table S1), brute-force recounts of Eq. H, exact closed forms of the two
decoupled limits (independent bonds; independent cells of six coupled arms,
enumerated), the infinite-temperature binomial, the frozen ground state,
brute-force Lennard-Jones sums, the representation counts r_3(n) of integers
as sums of three squares, Python's own lexicographic permutation order, and
the truncated Gamma law of the isobaric volume move.  No GPU is used.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import special

import oracle
from oracle import Oracle3

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers --
def _batch_mean(x, nbatch=50):
    x = np.asarray(x, dtype=np.float64)
    n = len(x) // nbatch * nbatch
    b = x[:n].reshape(nbatch, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nbatch)


def _arms(words):
    """[6, L, L, L] arm values of the words (sigma_a in bits [4a, 4a+3))
    indexed [z, y, x]."""
    w = np.asarray(words).astype(np.int64)
    return [(w >> (4 * a)) & 7 for a in range(6)]


def _counts_bruteforce(words, L):
    """N_HB_raw and N_sigma from the definitions of Eq. H on the cube: a bond
    joins arm 2k of a cell with arm 2k+1 of its neighbour one step along +axis
    k (x, y, z); N_sigma counts equal pairs among a cell's six arms."""
    w = np.asarray(words).reshape(L, L, L)
    arm = _arms(w)
    hb = int((arm[0] == np.roll(arm[1], -1, axis=2)).sum())
    hb += int((arm[2] == np.roll(arm[3], -1, axis=1)).sum())
    hb += int((arm[4] == np.roll(arm[5], -1, axis=0)).sum())
    co = 0
    for a in range(6):
        for b in range(a + 1, 6):
            co += int((arm[a] == arm[b]).sum())
    return hb, co


def _lj_bruteforce(v, epsilon=1.0, cutoff=6.0, box=7):
    """Per-cell LJ energy summed pair by pair: cell spacing r = v^(1/3),
    4 eps [(1/dist)^12 - (1/dist)^6] for every lattice vector with
    dist = r |d| < cutoff, half per cell."""
    r = v ** (1.0 / 3.0)
    total = 0.0
    for i in range(-box, box + 1):
        for j in range(-box, box + 1):
            for k in range(-box, box + 1):
                if i == j == k == 0:
                    continue
                dist = r * math.sqrt(i * i + j * j + k * k)
                if dist < cutoff:
                    total += 4.0 * epsilon * (dist ** -12 - dist ** -6)
    return 0.5 * total


def _random_words(rng, n, q):
    w = np.zeros(n, np.uint32)
    for a in range(6):
        w |= (rng.integers(0, q, n).astype(np.uint32) << np.uint32(4 * a))
    return w


# ---------------------------------------------------------------- layout --
def test_paper_layout_example_3d():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "paper_layout_example_3d.txt"))
            if l.strip() and not l.startswith("#")]
    kinds = {r[0] for r in rows}
    assert kinds == {"warp", "xyz", "pair"} and len(rows) == 23
    for r in rows:
        N, L = int(r[1]), int(r[2])
        assert L ** 3 == N
        if r[0] == "warp":
            cell, arm, idx = int(r[3]), int(r[4]), int(r[5])
            nb = oracle.neighbour3(L, cell, arm)
            assert (arm ^ 1) * N + nb == idx
            assert (nb == cell + 1) == (len(r) == 6)       # "wrap" marks the exceptions
        elif r[0] == "xyz":
            cell, x, y, z = map(int, r[3:7])
            # walking x, y, z steps along +x, +y, +z from cell 0 reaches the cell
            c = 0
            for arm, n in ((0, x), (2, y), (4, z)):
                for _ in range(n):
                    c = oracle.neighbour3(L, c, arm)
            assert c == cell
        else:
            ia, ib = int(r[3]), int(r[4])
            (aa, ca), (ab, cb) = divmod(ia, N), divmod(ib, N)
            assert ab == aa ^ 1
            assert oracle.neighbour3(L, ca, aa) == cb and oracle.neighbour3(L, cb, ab) == ca


@pytest.mark.parametrize("L", [2, 3, 5])
def test_neighbours_form_a_periodic_cube(L):
    N = L ** 3
    for c in range(N):
        for a in range(6):
            nb = oracle.neighbour3(L, c, a)
            assert 0 <= nb < N and oracle.neighbour3(L, nb, a ^ 1) == c
        # L steps along one axis come back to the cell
        for a in range(6):
            d = c
            for _ in range(L):
                d = oracle.neighbour3(L, d, a)
            assert d == c


# -------------------------------------------------------- Lennard-Jones --
def test_shell_multiplicities_are_r3():
    # r_3(n), the number of integer vectors with |d|^2 = n, for n = 1..14
    # (r_3(7) = 0: 7 is of the form 4^a (8b + 7) and not a sum of three squares)
    r3 = {1: 6, 2: 12, 3: 8, 4: 6, 5: 24, 6: 24, 8: 12, 9: 30, 10: 24, 11: 24, 12: 8,
          13: 24, 14: 48}
    d2, m = oracle.shell_table3(6.0)
    table = dict(zip(d2.tolist(), m.tolist()))
    for n, r in r3.items():
        assert table[n] == r
    assert 7 not in table and 15 not in table and 28 not in table
    # every lattice vector strictly inside radius 6, counted once
    g = np.arange(-6, 7)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    s = x * x + y * y + z * z
    assert int(((s > 0) & (s < 36)).sum()) == int(m.sum())


@pytest.mark.parametrize("v", [1.0, 1.03, 1.05, 2 ** 0.5, 1.7, 2.0, 2.6, 8.0, 30.0])
def test_lj3_cell_energy_matches_pairwise_sum(v):
    assert oracle.lj_cell_energy3(v) == pytest.approx(_lj_bruteforce(v), rel=1e-12, abs=1e-15)


def test_lj3_cutoff_edges():
    # shell |d|^2 = 35 leaves the cutoff when 35^3 v^2 >= 6^6
    v_edge = 216.0 / 35 ** 1.5
    below, above = oracle.lj_cell_energy3(v_edge * (1 - 1e-9)), oracle.lj_cell_energy3(v_edge * (1 + 1e-9))
    m35 = dict(zip(*[a.tolist() for a in oracle.shell_table3(6.0)]))[35]
    x = 1.0 / v_edge
    # the dropped shell's contribution 2 m (x^4/35^6 - x^2/35^3); the smooth part
    # of u moves by only ~1e-8 across the 2e-9 step in v
    assert below - above == pytest.approx(2 * m35 * (x ** 4 / 35 ** 6 - x ** 2 / 35 ** 3), rel=1e-4)


# ---------------------------------------------------- single-arm moves --
@pytest.mark.parametrize("L,q,g,kT", [(3, 3, 1, 0.7), (4, 6, 1, 0.45), (4, 6, 0, 0.45),
                                      (3, 2, 1, 1.3)])
def test_detailed_balance_against_recount(L, q, g, kT):
    """For sampled configurations, cells, arms and offsets: the move is
    reversible (the reverse offset maps back), its threshold is 2^32 min(1,
    exp(-dH/kT)) up to the 2^-32 floor, and dH from full recounts of both
    configurations (Eq. H with the gate) satisfies detailed balance."""
    p = oracle.params3(L=L, q=q, kT=kT, P=0.3)
    J_eff = p.J - p.P * p.v_HB
    rng = np.random.default_rng(L * 100 + q * 10 + g)
    N = L ** 3
    for trial in range(25):
        w = _random_words(rng, N, q)
        hb0, co0 = _counts_bruteforce(w, L)
        c = int(rng.integers(N))
        for a in range(6):
            s = (int(w[c]) >> (4 * a)) & 7
            seen = set()
            for k in range(q - 1):
                sp, T = oracle.arm_probe3(p, w, c, a, k, g)
                assert sp != s and sp < q
                seen.add(sp)
                w2 = w.copy()
                w2[c] = (int(w[c]) & ~(7 << (4 * a))) | (sp << (4 * a))
                hb1, co1 = _counts_bruteforce(w2, L)
                dH = -g * J_eff * (hb1 - hb0) - p.J_sigma * (co1 - co0)
                k_rev = (s - sp - 1) % q
                s_back, T_rev = oracle.arm_probe3(p, w2, c, a, k_rev, g)
                assert s_back == s
                pf, pr = T / 2 ** 32, T_rev / 2 ** 32
                assert pf == pytest.approx(min(1.0, math.exp(-dH / kT)), abs=2 ** -31)
                assert pf == pytest.approx(pr * math.exp(-dH / kT), abs=2 ** -30 * max(1.0, math.exp(-dH / kT)))
            assert len(seen) == q - 1   # the q-1 offsets reach the q-1 other states


# ------------------------------------------------------- exact limits --
def _cell_pairs_exact(q, beta_Js):
    """<pairs> of one cell of six arms with weight exp(beta J_sigma pairs),
    by enumeration of its q^6 configurations."""
    Z = E = 0.0
    for cfg in itertools.product(range(q), repeat=6):
        pairs = sum(cfg[a] == cfg[b] for a in range(6) for b in range(a + 1, 6))
        wgt = math.exp(beta_Js * pairs)
        Z += wgt
        E += pairs * wgt
    return E / Z


def test_independent_cells_limit():
    # J = 0 and v_HB = 0: the bonds drop out of Eq. H and every cell is an
    # independent 6-arm system weighted by exp(J_sigma N_sigma(cell) / kT)
    L, q, kT = 4, 3, 0.5
    p = oracle.params3(L=L, q=q, J=0.0, v_HB=0.0, kT=kT, volume_moves=0, seed=7)
    o = Oracle3(p)
    o.run(200)
    rec = o.run(6000, record_every=2)
    co = np.array([r["n_coop"] for r in rec], dtype=np.float64) / L ** 3
    m, se = _batch_mean(co)
    exact = _cell_pairs_exact(q, p.J_sigma / kT)
    assert abs(m - exact) < 5 * se, (m, se, exact)
    # the test resolves the coupling: the uncoupled value 15/q is far away
    assert abs(exact - 15 / q) > 20 * se


@pytest.mark.parametrize("g_liquid", [True, False])
def test_independent_bonds_limit(g_liquid):
    # J_sigma = 0: each of the 3N bonds is an independent pair of arms with
    # weight exp(g J_eff [equal] / kT), so <N_HB_raw> = 3N e^x / (e^x + q - 1)
    # with x = g J_eff / kT (the gas-like gate g = 0 gives 3N / q)
    L, q, kT = 4, 6, 0.6
    v0 = 1.5 if g_liquid else 2.5
    p = oracle.params3(L=L, q=q, J_sigma=0.0, kT=kT, P=0.1, v_iso_init=v0, volume_moves=0, seed=8)
    o = Oracle3(p)
    o.run(200)
    rec = o.run(6000, record_every=2)
    assert all(r["g"] == int(g_liquid) for r in rec)
    hb = np.array([r["n_hb_raw"] for r in rec], dtype=np.float64)
    x = (p.J - p.P * p.v_HB) / kT if g_liquid else 0.0
    exact = 3 * L ** 3 * math.exp(x) / (math.exp(x) + q - 1)
    m, se = _batch_mean(hb)
    assert abs(m - exact) < 5 * se, (m, se, exact)


def test_high_temperature_limit_binomial():
    # kT -> infinity: every proposal is accepted and the sigma stay iid
    # uniform: N_HB_raw ~ Binomial(3N, 1/q); N_sigma has mean 15N/q and
    # variance 15N (1/q)(1 - 1/q) (its 15N indicators are pairwise independent)
    L, q = 6, 6
    N = L ** 3
    p = oracle.params3(L=L, q=q, kT=1e300, volume_moves=0, seed=5)
    assert np.all(oracle.threshold_table3(p) == 2 ** 32)
    o = Oracle3(p)
    rec = o.run(6000, record_every=2)
    assert rec[-1]["acc_sigma"] == 6000 * 6 * N
    hb = np.array([r["n_hb_raw"] for r in rec], dtype=np.float64)
    co = np.array([r["n_coop"] for r in rec], dtype=np.float64)
    m, se = _batch_mean(hb)
    assert abs(m - 3 * N / q) < 5 * se
    assert abs(hb.var() / (3 * N / q * (1 - 1 / q)) - 1) < 0.15
    m, se = _batch_mean(co)
    assert abs(m - 15 * N / q) < 5 * se
    assert abs(co.var() / (15 * N / q * (1 - 1 / q)) - 1) < 0.15


@pytest.mark.parametrize("volume_moves", [0, 1])
def test_ground_state_is_frozen(volume_moves):
    # all sigma equal (every bond formed, all 15 pairs equal), liquid gate,
    # J_eff > 0, kT -> 0: every proposal loses a bond and five pairs and is
    # rejected; H = N u(v) - 3N J - 15N J_sigma + P (V_iso + 3N v_HB)
    L = 4
    N = L ** 3
    p = oracle.params3(L=L, q=6, kT=1e-3, init=oracle.INIT_ORDERED, volume_moves=volume_moves,
                       dv_max_frac=0.001)
    o = Oracle3(p)
    s0 = o.state()
    o.run(30)
    assert np.array_equal(o.state(), s0) and not s0.any()
    ob = o.observables()
    assert ob["n_hb_raw"] == 3 * N and ob["n_coop"] == 15 * N and ob["acc_sigma"] == 0
    v = ob["V_iso"] / N
    U = N * _lj_bruteforce(v)
    H = U - p.J * 3 * N - p.J_sigma * 15 * N + p.P * (ob["V_iso"] + p.v_HB * 3 * N)
    assert ob["U_LJ"] == pytest.approx(U, rel=1e-12)
    assert ob["H"] == pytest.approx(H, rel=1e-12)


# ------------------------------------------------------------ invariants --
@pytest.mark.parametrize("L", [3, 4, 5])
def test_incremental_counters_equal_recount(L):
    p = oracle.physical_params3(285.0, 20.0, L=L, seed=3, dv_max_frac=0.05)
    o = Oracle3(p)
    for _ in range(25):
        o.step()
        ob = o.observables()
        hb, co = _counts_bruteforce(o.w, L)
        assert (ob["n_hb_raw"], ob["n_coop"]) == (hb, co) == o.recount()
        assert sum(ob["n_state"]) == 6 * L ** 3


def test_random_init_is_uniform():
    L, q = 16, 6
    o = Oracle3(oracle.params3(L=L, q=q, seed=11))
    n = np.array(o.observables()["n_state"][:q], dtype=np.float64)
    e = 6 * L ** 3 / q
    assert ((n - e) ** 2 / e).sum() < 25     # chi^2, 5 degrees of freedom
    assert o.observables()["n_state"][q:] == [0] * (8 - q)


def test_checkpoint_resume_bit_exact():
    p = oracle.physical_params3(300.0, 0.1, L=5, seed=9, dv_max_frac=0.05)
    a = Oracle3(p)
    a.run(40)
    b = Oracle3(p)
    b.run(17)
    ob = b.observables()
    c = Oracle3(p, state=b.state(), V_iso=ob["V_iso"], sweep=ob["sweep"])
    c.run(23)
    oa, oc = a.observables(), c.observables()
    assert np.array_equal(a.state(), c.state())
    for k in ("sweep", "n_hb_raw", "n_coop", "V_iso", "H", "g"):
        assert oa[k] == oc[k]


# ----------------------------------------------------------- layer order --
def test_permutation_numbering_is_lexicographic():
    perms = list(itertools.permutations(range(6)))   # lexicographic order
    for i in range(720):
        assert tuple(oracle.permutation3(i)) == perms[i]


def test_layer_order_is_uniform():
    p = oracle.params3(seed=21)
    counts = np.zeros(720)
    index = {perm: i for i, perm in enumerate(itertools.permutations(range(6)))}
    for s in range(72000):
        counts[index[tuple(oracle.layer_order3(p, s))]] += 1
    chi2 = ((counts - 100) ** 2 / 100).sum()
    assert counts.min() > 0 and chi2 < 719 + 5 * math.sqrt(2 * 719)


# ------------------------------------------------------------ volume move --
def test_volume_move_truncated_gamma_3d():
    # J = J_sigma = v_HB = 0, LJ off: the weight of V_iso is V^N exp(-P V/kT)
    # on V >= N (hard core), mean (N+1) Q(N+2, bN) / (b Q(N+1, bN)), b = P/kT
    L = 2
    N = L ** 3
    for P, seed in ((0.5, 1), (3.0, 2)):
        p = oracle.params3(L=L, q=6, epsilon=0.0, J=0.0, J_sigma=0.0, v_HB=0.0, kT=1.0, P=P,
                           v_iso_init=1.5, dv_max_frac=0.4, seed=seed)
        V, acc = oracle.volume_chain3(p, N * 1.5, 0, 0, 400000)
        V = V[2000:]
        b = P / p.kT
        mean = (N + 1) * special.gammaincc(N + 2, b * N) / (b * special.gammaincc(N + 1, b * N))
        m, se = _batch_mean(V, 100)
        assert abs(m - mean) < 5 * se, (P, m, se, mean)
        assert V.min() >= N and 0 < acc < 400000


def test_volume_move_gate_term():
    # crossing the gate (v: 1.99 -> 2.01 and back) changes H by exactly
    # J_eff N_HB_raw times the gate change, on top of the LJ and PV terms:
    # the acceptance decided by the oracle agrees with exp(-dH/kT + N ln V'/V)
    p = oracle.params3(L=2, q=2, kT=0.8, P=0.2, v_iso_init=1.99, dv_max_frac=0.02, seed=4)
    N = 8
    J_eff = p.J - p.P * p.v_HB
    for step in range(200):
        V, acc = oracle.volume_chain3(p, N * 1.99, 5, step, 1)
        r = oracle.philox([0xFFFFFFFF, step, 0, 3], [p.seed, 0])
        u1 = ((int(r[0]) << 21) | (int(r[1]) >> 11)) * 2.0 ** -53
        u2 = ((int(r[2]) << 21) | (int(r[3]) >> 11)) * 2.0 ** -53
        V_new = N * 1.99 + (2 * u1 - 1) * p.dv_max_frac * N * p.v_iso_init
        g_new = 1 if V_new / N < 2 else 0
        dH = (N * (_lj_bruteforce(V_new / N) - _lj_bruteforce(1.99)) + p.P * (V_new - N * 1.99)
              - (g_new - 1) * J_eff * 5)
        arg = -dH / p.kT + N * math.log(V_new / (N * 1.99))
        if abs(u2 - math.exp(min(arg, 700))) < 1e-9:
            continue   # too close to call in a different summation order
        assert acc == (1 if u2 < math.exp(min(arg, 700)) else 0), step


@pytest.mark.parametrize("init", [oracle.INIT_RANDOM, oracle.INIT_ORDERED])
def test_window_init_run3_matches_whole_cube(init):
    """A box started by the init rule alone and run K layered steps agrees
    with the whole cube more than 2K + 2 cells inside (a pass moves
    information one cell along its axis, a step two)."""
    L, K = 24, 2
    op = oracle.physical_params3(300.0, 0.1, L=L, seed=19, init=init, dv_max_frac=0.05)
    ref = oracle.Oracle3(op)
    start = ref.state().copy()
    ob = ref.observables()
    V, _ = oracle.volume_chain3(op, ob["V_iso"], ob["n_hb_raw"], 0, K)
    gates = [int(v / L ** 3 < 2.0) for v in V]
    assert all(gg == ob["g"] for gg in gates)    # no gate change: the chain needs no bonds
    ref.run(K)
    whole = np.zeros(L ** 3, np.uint32)
    oracle.window_init_run3(op, whole, 0, 0, 0, L, L, L, 0, [])
    assert np.array_equal(whole.reshape(start.shape), start)
    w = np.zeros(L ** 3, np.uint32)
    x0, y0, z0, W, H, D = 2, 1, 3, 20, 21, 19
    oracle.window_init_run3(op, w, x0, y0, z0, W, H, D, 0, gates)
    m = 2 * K + 2
    cube = w.reshape(L, L, L)
    want = ref.state().reshape(L, L, L)
    inner = (slice(z0 + m, z0 + D - m), slice(y0 + m, y0 + H - m), slice(x0 + m, x0 + W - m))
    assert np.array_equal(cube[inner], want[inner])
    assert not cube[:z0].any()
