"""Pins of the 3D oracle (cubic lattice, six arms, layered schedule) against
what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the
indexing examples the paper prints for its N = 64 cubic lattice (Sec. II.C,
Table S1), brute-force recounts of Eq. H, exact closed forms of the two
decoupled limits (independent bonds; independent cells of six coupled arms,
enumerated), the infinite-temperature binomial, the frozen ground state,
brute-force Lennard-Jones sums, the representation counts r_3(n) of integers
as sums of three squares, Python's own lexicographic permutation order, and
the truncated Gamma law of the isobaric volume move.  The eta update of
App. A (checkerboard cubes, nine configurations) is pinned by an
enumeration of the perfect matchings of the cube graph written here from
coordinates, the partition of the edges into cubes, the invariant of exactly
two forbidden edges per molecule, detailed balance of the cube move against
brute-force recounts, and the decoupled limits with eta (2N allowed bonds).
No GPU is used.
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


def _cube_edges():
    """The twelve edges of the unit cube as (corner lo, corner hi, axis d),
    numbered e = 4 d + k: edge e runs along axis d from the k-th corner (in
    increasing corner number; corner j sits at offset (j & 1, j >> 1 & 1,
    j >> 2 & 1)) whose offset along d is 0."""
    edges = []
    for d in range(3):
        los = [j for j in range(8) if not (j >> d) & 1]
        for lo in los:
            edges.append((lo, lo | (1 << d), d))
    return edges


def _matchings_py():
    """The perfect matchings of the cube graph (four edges that cover each
    corner once), as 12-bit masks in increasing order, by trying every set
    of four edges."""
    edges = _cube_edges()
    out = []
    for comb in itertools.combinations(range(12), 4):
        cover = [0] * 8
        for e in comb:
            cover[edges[e][0]] += 1
            cover[edges[e][1]] += 1
        if all(c == 1 for c in cover):
            out.append(sum(1 << e for e in comb))
    return sorted(out)


def _eta_zero(L, cfg):
    """[z, y, x, d] True where the edge from cell (x, y, z) toward +axis d has
    eta = 0: cube (colour k, X, Y, Z) has its corner of smallest coordinates
    at (2X + k, 2Y + k, 2Z + k) and forbids the edges of its matching."""
    masks = _matchings_py()
    Hh = L // 2
    zero = np.zeros((L, L, L, 3), bool)
    edges = _cube_edges()
    for cube in range(2 * Hh ** 3):
        k, rem = divmod(cube, Hh ** 3)
        Z, rem = divmod(rem, Hh * Hh)
        Y, X = divmod(rem, Hh)
        cx, cy, cz = 2 * X + k, 2 * Y + k, 2 * Z + k
        m = masks[int(cfg[cube])]
        for e in range(12):
            if (m >> e) & 1:
                lo, _, d = edges[e]
                zero[(cz + (lo >> 2 & 1)) % L, (cy + (lo >> 1 & 1)) % L, (cx + (lo & 1)) % L, d] = True
    return zero


def _counts_eta(words, cfg, L):
    """N_HB_raw (bonded pairs on allowed edges) and N_sigma with eta."""
    w = np.asarray(words).reshape(L, L, L)
    arm = _arms(w)
    zero = _eta_zero(L, cfg)
    hb = int(((arm[0] == np.roll(arm[1], -1, axis=2)) & ~zero[..., 0]).sum())
    hb += int(((arm[2] == np.roll(arm[3], -1, axis=1)) & ~zero[..., 1]).sum())
    hb += int(((arm[4] == np.roll(arm[5], -1, axis=0)) & ~zero[..., 2]).sum())
    co = _counts_bruteforce(words, L)[1]
    return hb, co


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
    p = oracle.params3(L=L, q=q, kT=kT, P=0.3, eta_moves=0)
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


@pytest.mark.parametrize("eta_moves", [0, 1])
@pytest.mark.parametrize("g_liquid", [True, False])
def test_independent_bonds_limit(g_liquid, eta_moves):
    # J_sigma = 0: each allowed edge is an independent pair of arms with
    # weight exp(g J_eff [equal] / kT) (a forbidden edge weighs q^2 whatever
    # its arms), so <N_HB_raw> = n e^x / (e^x + q - 1) with x = g J_eff / kT:
    # n = 3N allowed edges with eta = 1 everywhere, n = 2N with the eta of
    # App. A (every configuration forbids exactly N edges, so all are equally
    # weighted); the gas-like gate g = 0 gives n / q
    L, q, kT = 4, 6, 0.6
    v0 = 1.5 if g_liquid else 2.5
    p = oracle.params3(L=L, q=q, J_sigma=0.0, kT=kT, P=0.1, v_iso_init=v0, volume_moves=0, seed=8,
                       eta_moves=eta_moves)
    o = Oracle3(p)
    o.run(200)
    rec = o.run(6000, record_every=2)
    assert all(r["g"] == int(g_liquid) for r in rec)
    hb = np.array([r["n_hb_raw"] for r in rec], dtype=np.float64)
    x = (p.J - p.P * p.v_HB) / kT if g_liquid else 0.0
    n = (2 if eta_moves else 3) * L ** 3
    exact = n * math.exp(x) / (math.exp(x) + q - 1)
    m, se = _batch_mean(hb)
    assert abs(m - exact) < 5 * se, (m, se, exact)


def test_eta_configurations_uniform_when_bonds_decouple():
    # J_sigma = 0: the weight of a cube configuration does not depend on
    # which four edges it forbids (above), so in the long run each of the
    # nine is taken equally often (chi^2 over cube-steps, 8 degrees of freedom
    # per sample, samples 10 steps apart)
    L, q, kT = 4, 6, 0.6
    p = oracle.params3(L=L, q=q, J_sigma=0.0, kT=kT, P=0.1, v_iso_init=1.5, volume_moves=0, seed=12)
    o = Oracle3(p)
    o.run(100)
    counts = np.zeros(9)
    for _ in range(600):
        o.run(10)
        counts += np.bincount(o.eta(), minlength=9)
    e = counts.sum() / 9
    chi2 = ((counts - e) ** 2 / e).sum()
    assert chi2 < 8 + 6 * math.sqrt(16) + 10, (counts, chi2)


@pytest.mark.parametrize("eta_moves", [0, 1])
def test_high_temperature_limit_binomial(eta_moves):
    # kT -> infinity: every proposal is accepted and the sigma stay iid
    # uniform: N_HB_raw ~ Binomial(n, 1/q) over the n allowed edges (3N, or
    # 2N with the eta of App. A); N_sigma has mean 15N/q and variance 15N
    # (1/q)(1 - 1/q) (its 15N indicators are pairwise independent)
    L, q = 6, 6
    N = L ** 3
    p = oracle.params3(L=L, q=q, kT=1e300, volume_moves=0, seed=5, eta_moves=eta_moves)
    assert np.all(oracle.threshold_table3(p) == 2 ** 32)
    assert np.all(oracle.eta_table3(p) == 2 ** 32)
    o = Oracle3(p)
    rec = o.run(6000, record_every=2)
    assert rec[-1]["acc_sigma"] == 6000 * 6 * N
    if eta_moves:
        assert o.acc_eta == 6000 * N // 4
    n = (2 if eta_moves else 3) * N
    hb = np.array([r["n_hb_raw"] for r in rec], dtype=np.float64)
    co = np.array([r["n_coop"] for r in rec], dtype=np.float64)
    m, se = _batch_mean(hb)
    assert abs(m - n / q) < 5 * se
    assert abs(hb.var() / (n / q * (1 - 1 / q)) - 1) < 0.15
    m, se = _batch_mean(co)
    assert abs(m - 15 * N / q) < 5 * se
    assert abs(co.var() / (15 * N / q * (1 - 1 / q)) - 1) < 0.15


@pytest.mark.parametrize("volume_moves,eta_moves", [(0, 0), (1, 0), (1, 1)])
def test_ground_state_is_frozen(volume_moves, eta_moves):
    # all sigma equal (every bond formed, all 15 pairs equal), liquid gate,
    # J_eff > 0, kT -> 0: every sigma proposal loses five pairs (and a bond on
    # an allowed edge) and is rejected; H = N u(v) - n J - 15N J_sigma + P
    # (V_iso + n v_HB) with n = 3N bonds (2N with eta).  With eta every cube
    # move trades four bonded edges for four bonded edges (dN_HB = 0) and is
    # accepted every step.
    L = 4
    N = L ** 3
    p = oracle.params3(L=L, q=6, kT=1e-3, init=oracle.INIT_ORDERED, volume_moves=volume_moves,
                       dv_max_frac=0.001, eta_moves=eta_moves)
    o = Oracle3(p)
    s0 = o.state()
    o.run(30)
    assert np.array_equal(o.state(), s0) and not s0.any()
    ob = o.observables()
    nb = (2 if eta_moves else 3) * N
    assert ob["n_hb_raw"] == nb and ob["n_coop"] == 15 * N and ob["acc_sigma"] == 0
    if eta_moves:
        assert o.acc_eta == 30 * N // 4
    v = ob["V_iso"] / N
    U = N * _lj_bruteforce(v)
    H = U - p.J * nb - p.J_sigma * 15 * N + p.P * (ob["V_iso"] + p.v_HB * nb)
    assert ob["U_LJ"] == pytest.approx(U, rel=1e-12)
    assert ob["H"] == pytest.approx(H, rel=1e-12)


# ------------------------------------------------------------ invariants --
@pytest.mark.parametrize("L,eta_moves", [(3, 0), (4, 0), (5, 0), (4, 1), (6, 1)])
def test_incremental_counters_equal_recount(L, eta_moves):
    p = oracle.physical_params3(285.0, 20.0, L=L, seed=3, dv_max_frac=0.05, eta_moves=eta_moves)
    o = Oracle3(p)
    for _ in range(25):
        o.step()
        ob = o.observables()
        if eta_moves:
            hb, co = _counts_eta(o.w, o.eta(), L)
        else:
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


@pytest.mark.parametrize("L,eta_moves", [(5, 0), (6, 1)])
def test_checkpoint_resume_bit_exact(L, eta_moves):
    p = oracle.physical_params3(300.0, 0.1, L=L, seed=9, dv_max_frac=0.05, eta_moves=eta_moves)
    a = Oracle3(p)
    a.run(40)
    b = Oracle3(p)
    b.run(17)
    ob = b.observables()
    c = Oracle3(p, state=b.state(), V_iso=ob["V_iso"], sweep=ob["sweep"], eta=b.eta())
    c.run(23)
    oa, oc = a.observables(), c.observables()
    assert np.array_equal(a.state(), c.state())
    assert np.array_equal(a.eta(), c.eta())
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


@pytest.mark.parametrize("eta_moves", [0, 1])
@pytest.mark.parametrize("init", [oracle.INIT_RANDOM, oracle.INIT_ORDERED])
def test_window_init_run3_matches_whole_cube(init, eta_moves):
    """A box started by the init rule alone and run K layered steps agrees
    with the whole cube more than 2K + 2 cells inside (a pass moves
    information one cell along its axis, a step two), 3K + 2 with eta
    moves (a cube move carries it one cell more)."""
    L, K = 24, 2
    op = oracle.physical_params3(300.0, 0.1, L=L, seed=19, init=init, dv_max_frac=0.05,
                                 eta_moves=eta_moves)
    ref = oracle.Oracle3(op)
    start = ref.state().copy()
    ob = ref.observables()
    V, _ = oracle.volume_chain3(op, ob["V_iso"], ob["n_hb_raw"], 0, K)
    gates = [int(v / L ** 3 < 2.0) for v in V]
    assert all(gg == ob["g"] for gg in gates)    # no gate change: the chain needs no bonds
    ref.run(K)
    whole = np.zeros(L ** 3, np.uint32)
    eta_whole = np.zeros(L ** 3 // 4, np.uint8)
    oracle.window_init_run3(op, whole, 0, 0, 0, L, L, L, 0, [], eta_whole)
    assert np.array_equal(whole.reshape(start.shape), start)
    w = np.zeros(L ** 3, np.uint32)
    eta_w = np.zeros(L ** 3 // 4, np.uint8)
    x0, y0, z0, W, H, D = 2, 1, 3, 20, 21, 19
    oracle.window_init_run3(op, w, x0, y0, z0, W, H, D, 0, gates, eta_w)
    m = (3 if eta_moves else 2) * K + 2
    cube = w.reshape(L, L, L)
    want = ref.state().reshape(L, L, L)
    inner = (slice(z0 + m, z0 + D - m), slice(y0 + m, y0 + H - m), slice(x0 + m, x0 + W - m))
    assert np.array_equal(cube[inner], want[inner])
    assert not cube[:z0].any()


# ------------------------------------------------------------- eta (App. A) --
def test_nine_configurations_are_the_cube_matchings():
    """App. A's nine configurations: the oracle's list equals the perfect
    matchings of the cube graph found here by trying all 495 sets of four
    edges, and there are exactly nine of them."""
    n, masks = oracle.matchings3()
    assert n == 9
    assert masks == _matchings_py()
    edges = _cube_edges()
    for m in masks:   # every corner loses exactly one of its three edges
        for j in range(8):
            assert sum(1 for e in range(12) if (m >> e) & 1 and j in edges[e][:2]) == 1


@pytest.mark.parametrize("L", [2, 4, 6])
def test_checkerboard_cubes_partition_the_edges(L):
    """Every molecule is a corner of exactly one cube of each colour, and the
    (cube, edge number) of the oracle's edge lookup runs over each of the 3N
    edges exactly once, consistent with the cubes' corner cells."""
    N = L ** 3
    ncube = N // 4
    member = np.zeros((N, 2), np.int64)
    for cube in range(ncube):
        cells = oracle.cube_corner_cells3(L, cube)
        assert len(set(cells)) == (8 if L > 1 else 1)
        for c in cells:
            member[c, cube // (ncube // 2)] += 1
    assert (member == 1).all()
    seen = set()
    edges = _cube_edges()
    for c in range(N):
        for a in range(6):
            cube, e = oracle.edge_of3(L, c, a)
            lo, hi, d = edges[e]
            assert d == a // 2
            cells = oracle.cube_corner_cells3(L, cube)
            nb = oracle.neighbour3(L, c, a)
            # the edge joins c and its neighbour in direction a, in that cube
            assert {cells[lo], cells[hi]} == {c, nb} or (L == 2 and {cells[lo], cells[hi]} == {c, nb})
            if a % 2 == 0:
                assert cells[lo] == c
            else:
                assert cells[hi] == c
            seen.add((cube, e))
    assert len(seen) == 3 * N == 12 * ncube


@pytest.mark.parametrize("init", [oracle.INIT_RANDOM, oracle.INIT_ORDERED])
def test_every_molecule_keeps_two_forbidden_edges(init):
    """After every step each molecule has exactly two of its six edges with
    eta = 0 (so at most four bonds, Sec. II.A), read both from the oracle's
    per-arm lookup and from the cube configurations directly."""
    L = 6
    p = oracle.physical_params3(300.0, 0.1, L=L, seed=13, init=init)
    o = Oracle3(p)
    for _ in range(12):
        o.step()
        zero = _eta_zero(L, o.eta())
        per_cell = zero.sum(axis=3)
        per_cell = per_cell + np.roll(zero[..., 0], 1, axis=2) + np.roll(zero[..., 1], 1, axis=1) \
            + np.roll(zero[..., 2], 1, axis=0)
        assert (per_cell == 2).all()
        eta = o.eta()
        for c in range(0, L ** 3, 7):
            assert sum(1 - oracle.eta_of3(p, eta, c, a) for a in range(6)) == 2
    assert o.acc_eta > 0


@pytest.mark.parametrize("g,kT", [(1, 0.45), (1, 1.2), (0, 0.45)])
def test_cube_move_detailed_balance(g, kT):
    """For sampled sigma and cube configurations, every cube and every offset:
    the proposal is one of the eight other configurations (the eight offsets
    reach all of them), the reverse offset maps back, dN_HB equals the change
    of a brute-force recount, and the threshold is 2^32 min(1, exp(-dH/kT))
    with dH = -g J_eff dN_HB, so P(a -> b) exp(-H_a/kT) = P(b -> a)
    exp(-H_b/kT) to the 2^-32 resolution."""
    L, q = 4, 3
    p = oracle.params3(L=L, q=q, kT=kT, P=0.3)
    J_eff = p.J - p.P * p.v_HB
    rng = np.random.default_rng(int(kT * 100) + g)
    N = L ** 3
    for trial in range(6):
        w = _random_words(rng, N, q)
        cfg = rng.integers(0, 9, N // 4).astype(np.uint8)
        hb0, _ = _counts_eta(w, cfg, L)
        for cube in rng.choice(N // 4, 4, replace=False):
            reached = set()
            for k in range(8):
                nw, dhb, T = oracle.eta_probe3(p, w, cfg, int(cube), k, g)
                assert nw != cfg[cube] and 0 <= nw < 9
                reached.add(nw)
                cfg2 = cfg.copy()
                cfg2[cube] = nw
                hb1, _ = _counts_eta(w, cfg2, L)
                assert dhb == hb1 - hb0
                dH = -g * J_eff * dhb
                k_rev = (int(cfg[cube]) - nw - 1) % 9
                back, dhb_rev, T_rev = oracle.eta_probe3(p, w, cfg2, int(cube), k_rev, g)
                assert back == cfg[cube] and dhb_rev == -dhb
                pf, pr = T / 2 ** 32, T_rev / 2 ** 32
                assert pf == pytest.approx(min(1.0, math.exp(-dH / kT)), abs=2 ** -31)
                assert pf == pytest.approx(pr * math.exp(-dH / kT),
                                           abs=2 ** -30 * max(1.0, math.exp(-dH / kT)))
            assert len(reached) == 8


def test_eta_moves_follow_the_step_draws():
    """The cube moves of one step use Philox((cube, step, 5)): offset
    floor(r0 8 / 2^32), acceptance word r1 (recomputed here from the oracle's
    Philox and its probe), and leave the sigma alone."""
    L = 4
    p = oracle.physical_params3(300.0, 0.1, L=L, seed=33, volume_moves=0)
    o = Oracle3(p)
    o.run(3)
    w, cfg = o.w.copy(), o.eta()
    g = o.observables()["g"]
    want = cfg.copy()
    for cube in range(L ** 3 // 4):
        r = oracle.philox([cube, 3, 0, 5], [p.seed & 0xFFFFFFFF, p.seed >> 32])
        k = (int(r[0]) * 8) >> 32
        nw, _, T = oracle.eta_probe3(p, w, cfg, cube, k, g)
        if int(r[1]) < T:
            want[cube] = nw
    o.eta_moves()
    assert np.array_equal(o.eta(), want) and np.array_equal(o.w, w)


def test_random_eta_init_is_uniform():
    L = 24
    o = Oracle3(oracle.params3(L=L, q=6, seed=17))
    counts = np.bincount(o.eta(), minlength=9).astype(np.float64)
    e = counts.sum() / 9
    assert ((counts - e) ** 2 / e).sum() < 8 + 5 * 4
    assert not Oracle3(oracle.params3(L=L, q=6, seed=17, init=oracle.INIT_ORDERED)).eta().any()


def test_eta_needs_an_even_side():
    with pytest.raises(ValueError):
        Oracle3(oracle.params3(L=5, q=6))
    Oracle3(oracle.params3(L=5, q=6, eta_moves=0))
