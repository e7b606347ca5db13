/*
 * cvf_oracle3.c -- plain CPU oracle of the paper's own 3D CVF Metropolis
 * (arXiv:2505.05919, Sec. II): a periodic cubic lattice of N = L^3 cells,
 * six bonding indices per cell, the layered partition of Sec. II.C (the six
 * arm domains updated one after the other, in an order drawn every MC step),
 * Eq. (H) with up to C(6,2) = 15 cooperative pairs per cell, and the isobaric
 * volume move of Sec. II.B with the Lennard-Jones sum of the cubic lattice.
 *
 * TEST INFRASTRUCTURE, like cvf_oracle.c: only tests/, smoke() and the CPU
 * legs of bench.py use it; it shares no code with the CUDA library.  Every
 * step is written in the order of the paper, one variable at a time.
 *
 * Readings (besides the 2D oracle's, which carry over):
 *   - state: one uint32 word per cell, sigma of arm a in bits [4a, 4a+3)
 *     (one nibble per arm, bit 4a+3 and bits 24..31 zero);
 *   - cell c = x + L (y + L z) and arms 0..5 = left, right, front, back,
 *     top, bottom (Sec. II.C; the cell coordinates of Table S1).  The
 *     coalescing example of Sec. II.C (left arms of cells 0..15 meet the
 *     right arms of cells 1..16) puts arm 0 at +x, and Table S1's covalent
 *     pair (257, 337) joins the top arm of cell (1,0,0) with the bottom arm
 *     of cell (1,0,1), so arm 4 points to +z; arm 2 points to +y by the same
 *     pattern (the paper prints no y example), and arm a ^ 1 is the
 *     opposite of arm a;
 *   - eta (App. A, with eta_moves = 1): the checkerboard cubes are the unit
 *     cells whose corner of smallest coordinates has all three coordinates
 *     even (colour 0) or all odd (colour 1); every molecule is a corner of
 *     one cube of each colour and every edge lies in exactly one cube, so
 *     the L^3/4 cubes (L even) partition the 3N edges.  A cube's eta = 0
 *     edges are one of the nine perfect matchings of the cube graph (each
 *     corner loses exactly one of its three edges in the cube, so every
 *     molecule keeps four allowed bonds whatever the other cubes do: the
 *     nine configurations of App. A), numbered 0..8 in increasing order of
 *     their 12-bit edge mask.  The eta step of an MC step moves every cube
 *     by Metropolis: configuration (c + 1 + k) mod 9 with k = floor(r0 8 /
 *     2^32), accepted iff r1 < T[g][dN_HB + 4], T from dH = -g J_eff dN_HB
 *     (N_HB is the only term of Eq. H that involves eta), r = Philox((cube,
 *     step, 5)); the cubes share no edge, so they move together.  Random
 *     init: configuration floor(r0 9 / 2^32), r = Philox((cube, 0, 0, 6));
 *     ordered init: configuration 0.  With eta_moves = 0, eta = 1 for every
 *     pair (up to six bonds per molecule);
 *   - one MC step: volume move, then eta, then six passes, pass i updating arm
 *     order[i] of every cell; order is permutation number
 *     floor(w 720 / 2^32) of the six arms in lexicographic order, w word 0
 *     of Philox((2^32-2, step, 4));
 *   - random numbers: the draw of arm a of cell c in step s is word c mod 4
 *     of Philox((floor(c / 4), s, 8 + a)); w (q-1) = k 2^32 + u gives the
 *     proposal offset k and the acceptance draw u; the random initial state
 *     is sigma_a(c) = floor(w q / 2^32), w word c mod 4 of
 *     Philox((floor(c / 4), 0, 16 + a));
 *   - Lennard-Jones: r = v_iso^(1/3) (Sec. II.A), so a pair at lattice
 *     vector d is at distance r |d| and (r0 / dist)^6 = 1 / (|d|^6 v^2); it
 *     lies inside the 6 r0 cutoff iff |d|^6 v^2 < 6^6 (no cube roots); per
 *     cell u(v) = 1/2 sum over those pairs of 4 eps [(r0/dist)^12 -
 *     (r0/dist)^6], taken pair by pair, shell by shell in increasing |d|^2;
 *   - the gate is liquid iff v_iso < 2 (Sec. II.A, gas-like when
 *     v_iso >= 2 v0).
 * Compile: gcc -O2 -std=c11 -ffp-contract=off (with cvf_oracle.c).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "cvf_oracle.h"

static uint32_t o3_arm(uint32_t w, int a) { return (w >> (4 * a)) & 7u; }

static void o3_philox(const orc_params *p, uint32_t word0, int64_t step, uint32_t tag,
                      uint32_t out[4]) {
  uint32_t ctr[4] = {word0, (uint32_t)((uint64_t)step & 0xFFFFFFFFu),
                     (uint32_t)((uint64_t)step >> 32), tag};
  uint32_t key[2] = {(uint32_t)(p->seed & 0xFFFFFFFFu), (uint32_t)(p->seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

static uint32_t o3_scale(uint32_t w, uint32_t n) {
  return (uint32_t)(((uint64_t)w * (uint64_t)n) >> 32);
}

/* The random word of (cell c, tag) in step `step`: word c mod 4 of the
   Philox block of counter (c / 4, step, tag). */
static uint32_t o3_word(const orc_params *p, int64_t c, int64_t step, uint32_t tag) {
  uint32_t r[4];
  o3_philox(p, (uint32_t)(c / 4), step, tag, r);
  return r[c % 4];
}

int64_t orc3_neighbour(int32_t L, int64_t c, int arm) {
  int64_t x = c % L, y = (c / L) % L, z = c / ((int64_t)L * L);
  switch (arm) {
    case 0: x = (x + 1) % L; break;
    case 1: x = (x + L - 1) % L; break;
    case 2: y = (y + 1) % L; break;
    case 3: y = (y + L - 1) % L; break;
    case 4: z = (z + 1) % L; break;
    default: z = (z + L - 1) % L; break;
  }
  return (z * L + y) * L + x;
}

/* ---------------------------------------------------------------- LJ 3D --- */
/* Shells of the cubic lattice inside the cutoff at the hard-core density:
   squared lengths |d|^2 < cutoff^2 (ascending) and their multiplicities,
   counted by brute force over a cube of lattice vectors. */
int orc3_shell_table(double cutoff, int64_t *d2s, int64_t *mult, int cap) {
  int R = (int)ceil(cutoff) + 1;
  int64_t maxd2 = (int64_t)(cutoff * cutoff) + 1;
  int n = 0;
  for (int64_t d2 = 1; d2 <= maxd2; ++d2) {
    if (!((double)d2 < cutoff * cutoff)) continue;
    int64_t m = 0;
    for (int i = -R; i <= R; ++i)
      for (int j = -R; j <= R; ++j)
        for (int k = -R; k <= R; ++k)
          if ((int64_t)i * i + (int64_t)j * j + (int64_t)k * k == d2) ++m;
    if (m > 0) {
      if (n >= cap) return -1;
      d2s[n] = d2;
      mult[n] = m;
      ++n;
    }
  }
  return n;
}

#define O3_MAX_SHELLS 1024
double orc3_lj_cell_energy(double v_iso, double epsilon, double cutoff) {
  static int64_t d2s[O3_MAX_SHELLS], mult[O3_MAX_SHELLS];
  static double last_cutoff = -1.0;
  static int n = 0;
  if (cutoff != last_cutoff) {
    n = orc3_shell_table(cutoff, d2s, mult, O3_MAX_SHELLS);
    if (n < 0) n = 0;
    last_cutoff = cutoff;
  }
  double rc6 = cutoff * cutoff * cutoff * cutoff * cutoff * cutoff;
  double sum = 0.0;
  for (int s = 0; s < n; ++s) {
    double d6v2 = (double)(d2s[s] * d2s[s] * d2s[s]) * v_iso * v_iso; /* (dist / r0)^6 */
    if (!(d6v2 < rc6)) break; /* shells ascend: the rest lie outside */
    double y6 = 1.0 / d6v2;   /* (r0 / dist)^6 */
    double y12 = y6 * y6;     /* (r0 / dist)^12 */
    double pair = (4.0 * epsilon) * (y12 - y6);
    sum += (double)mult[s] * pair;
  }
  return 0.5 * sum;
}

/* ------------------------------------------------------------ thresholds -- */
/* [g][dN_HB + 1][dN_sigma + 5]: dN_sigma in -5..5 (five other arms). */
void orc3_threshold_table(const orc_params *p, uint64_t out[2][3][11]) {
  double J_eff = p->J - p->P * p->v_HB;
  for (int g = 0; g < 2; ++g)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 11; ++j) {
        int dhb = i - 1, dc = j - 5;
        double dH = -((double)g * J_eff) * (double)dhb - p->J_sigma * (double)dc;
        out[g][i][j] = (dH <= 0.0) ? ((uint64_t)1 << 32)
                                   : (uint64_t)(exp(-dH / p->kT) * 4294967296.0);
      }
}

/* ------------------------------------------------------------------ eta -- */
#define O3_TAG_ETA 5u
#define O3_TAG_ETA_INIT 6u

/* Edge e (0..11) of a cube runs along axis d = e / 4 from corner lo to corner
   lo | (1 << d), lo the (e % 4)-th of the four corners with bit d clear in
   increasing order; corner j sits at offset (j & 1, (j >> 1) & 1, (j >> 2) &
   1) from the cube's corner of smallest coordinates. */
static int o3_edge_lo(int e) {
  int d = e / 4, k = e % 4, n = 0;
  for (int j = 0; j < 8; ++j)
    if (!((j >> d) & 1)) {
      if (n == k) return j;
      ++n;
    }
  return -1;
}

/* The nine configurations: the 12-bit masks of the perfect matchings of the
   cube graph (four edges covering each of the eight corners once), in
   increasing order.  Returns how many there are. */
int orc3_matchings(uint16_t out[9]) {
  int n = 0;
  for (int m = 0; m < 4096; ++m) {
    int cover[8] = {0, 0, 0, 0, 0, 0, 0, 0}, edges = 0;
    for (int e = 0; e < 12; ++e)
      if ((m >> e) & 1) {
        int lo = o3_edge_lo(e);
        cover[lo] += 1;
        cover[lo | (1 << (e / 4))] += 1;
        ++edges;
      }
    int ok = (edges == 4);
    for (int j = 0; j < 8; ++j) ok = ok && (cover[j] == 1);
    if (ok) {
      if (n < 9) out[n] = (uint16_t)m;
      ++n;
    }
  }
  return n;
}

static uint16_t o3_mask(uint8_t cfg) {
  static uint16_t masks[9];
  static int ready = 0;
  if (!ready) {
    orc3_matchings(masks);
    ready = 1;
  }
  return masks[cfg];
}

static int64_t o3_mod(int64_t a, int64_t L) { return ((a % L) + L) % L; }

/* Cube index: colour (L/2)^3 + (Z (L/2) + Y) (L/2) + X for the cube whose
   corner of smallest coordinates is (2X + colour, 2Y + colour, 2Z + colour). */
static int64_t o3_cube_index(int32_t L, int64_t cx, int64_t cy, int64_t cz) {
  int64_t H = L / 2, colour = cx & 1;
  return ((colour * H + (cz >> 1)) * H + (cy >> 1)) * H + (cx >> 1);
}

void orc3_cube_corner_cells(int32_t L, int64_t cube, int64_t cells[8]) {
  int64_t H = L / 2;
  int64_t X = cube % H, Y = (cube / H) % H, Z = (cube / (H * H)) % H, colour = cube / (H * H * H);
  int64_t cx = 2 * X + colour, cy = 2 * Y + colour, cz = 2 * Z + colour;
  for (int j = 0; j < 8; ++j) {
    int64_t x = (cx + (j & 1)) % L, y = (cy + ((j >> 1) & 1)) % L, z = (cz + ((j >> 2) & 1)) % L;
    cells[j] = (z * L + y) * L + x;
  }
}

/* The cube holding the edge of arm a of cell c, and the edge's number in it.
   The edge joins v (its end of smaller coordinate along axis d = a / 2: c
   itself for a +d arm, the neighbour for a -d arm) and v + e_d; the cube's
   corner has v's coordinate along d and, along each other axis, v's
   coordinate or the one below, whichever has the parity of v_d. */
void orc3_edge_of(int32_t L, int64_t c, int a, int64_t *cube, int *e) {
  int d = a >> 1;
  int64_t v = (a & 1) ? orc3_neighbour(L, c, a) : c;
  int64_t vc[3] = {v % L, (v / L) % L, v / ((int64_t)L * L)};
  int64_t cc[3];
  int j = 0;
  for (int u = 0; u < 3; ++u) {
    if (u == d) {
      cc[u] = vc[u];
    } else if (((vc[u] - vc[d]) & 1) == 0) {
      cc[u] = vc[u];
    } else {
      cc[u] = o3_mod(vc[u] - 1, L);
      j |= 1 << u;
    }
  }
  *cube = o3_cube_index(L, cc[0], cc[1], cc[2]);
  int k = 0;
  for (int i = 0; i < 8; ++i)
    if (!((i >> d) & 1)) {
      if (i == j) break;
      ++k;
    }
  *e = 4 * d + k;
}

/* eta of the edge of arm a of cell c: 0 if the edge is in its cube's
   matching, else 1; always 1 without eta moves. */
int orc3_eta_of(const orc_params *p, const uint8_t *eta, int64_t c, int a) {
  if (!p->eta_moves || !eta) return 1;
  int64_t cube;
  int e;
  orc3_edge_of(p->L, c, a, &cube, &e);
  return ((o3_mask(eta[cube]) >> e) & 1) ? 0 : 1;
}

/* Thresholds of a cube move, [g][dN_HB + 4]: dH = -g J_eff dN_HB (the eta
   enter Eq. H only through N_HB; the P v_HB N_HB of P V is in J_eff), T =
   2^32 if dH <= 0, else floor(exp(-dH / kT) 2^32). */
void orc3_eta_table(const orc_params *p, uint64_t out[2][9]) {
  double J_eff = p->J - p->P * p->v_HB;
  for (int g = 0; g < 2; ++g)
    for (int i = 0; i < 9; ++i) {
      int dhb = i - 4;
      double dH = -((double)g * J_eff) * (double)dhb;
      out[g][i] = (dH <= 0.0) ? ((uint64_t)1 << 32)
                              : (uint64_t)(exp(-dH / p->kT) * 4294967296.0);
    }
}

/* The 12-bit mask of the bonded edges of a cube: bit e set when the +d arm
   of corner lo and the -d arm of corner lo | (1 << d) are equal. */
static uint16_t o3_cube_bonds(int32_t L, const uint32_t *w, int64_t cube) {
  int64_t cells[8];
  orc3_cube_corner_cells(L, cube, cells);
  uint16_t b = 0;
  for (int e = 0; e < 12; ++e) {
    int d = e / 4, lo = o3_edge_lo(e), hi = lo | (1 << d);
    if (o3_arm(w[cells[lo]], 2 * d) == o3_arm(w[cells[hi]], 2 * d + 1)) b |= (uint16_t)(1u << e);
  }
  return b;
}

static int o3_popc12(uint16_t m) {
  int n = 0;
  for (int e = 0; e < 12; ++e) n += (m >> e) & 1;
  return n;
}

/* Decision data of the move of cube `cube` with proposal offset k (0..7)
   on an explicit configuration: the proposed configuration, the change of
   N_HB_raw and the threshold. */
void orc3_eta_probe(const orc_params *p, const uint32_t *w, const uint8_t *eta,
                    int64_t cube, uint32_t k, int32_t g, uint32_t *cfg_new,
                    int32_t *dhb, uint64_t *T) {
  uint64_t table[2][9];
  orc3_eta_table(p, table);
  uint16_t b = o3_cube_bonds(p->L, w, cube);
  uint8_t old = eta[cube];
  uint8_t nw = (uint8_t)((old + 1u + k) % 9u);
  /* the edges leaving the matching become allowed bonds, the edges entering
     it stop counting */
  int d = o3_popc12((uint16_t)(b & o3_mask(old))) - o3_popc12((uint16_t)(b & o3_mask(nw)));
  *cfg_new = nw;
  *dhb = d;
  *T = table[g][d + 4];
}

/* Step 2 of the MC step (Sec. II.B, App. A): every cube makes one
   Metropolis move of its configuration with the sigma fixed. */
void orc3_eta_moves(orc3_state *st) {
  const orc_params *p = &st->p;
  for (int64_t cube = 0; cube < st->ncube; ++cube) {
    uint32_t r[4];
    o3_philox(p, (uint32_t)cube, st->sweep, O3_TAG_ETA, r);
    uint32_t k = o3_scale(r[0], 8u), nw;
    int32_t dhb;
    uint64_t T;
    orc3_eta_probe(p, st->w, st->eta, cube, k, st->g, &nw, &dhb, &T);
    if ((uint64_t)r[1] < T) {
      st->eta[cube] = (uint8_t)nw;
      st->n_hb_raw += dhb;
      st->acc_eta += 1;
    }
  }
}

/* N_HB_raw with the eta: bonds of the +axis arms whose edge is allowed. */
void orc3_recount_eta(const orc_params *p, const uint32_t *w, const uint8_t *eta,
                      int64_t *n_hb_raw, int64_t *n_coop) {
  int64_t N = (int64_t)p->L * p->L * p->L, hb = 0, co = 0;
  for (int64_t c = 0; c < N; ++c) {
    uint32_t wc = w[c];
    for (int a = 0; a < 6; a += 2)
      if (o3_arm(wc, a) == o3_arm(w[orc3_neighbour(p->L, c, a)], a + 1) &&
          orc3_eta_of(p, eta, c, a))
        ++hb;
    for (int a = 0; a < 6; ++a)
      for (int b = a + 1; b < 6; ++b)
        if (o3_arm(wc, a) == o3_arm(wc, b)) ++co;
  }
  *n_hb_raw = hb;
  *n_coop = co;
}

/* The initial configuration of a cube: 0 (ordered init) or floor(r0 9 /
   2^32) with r = Philox((cube, 0, 0, 6)) (random init). */
static uint8_t o3_eta_init_cfg(const orc_params *p, int64_t cube) {
  if (p->init != ORC_INIT_RANDOM) return 0;
  uint32_t r[4];
  o3_philox(p, (uint32_t)cube, 0, O3_TAG_ETA_INIT, r);
  return (uint8_t)o3_scale(r[0], 9u);
}

/* ----------------------------------------------------------------- state -- */
/* Full count: bonds between arm a of c and arm a^1 of its neighbour (each
   bond once, from its +axis end) and the equal pairs among a cell's six
   arms. */
void orc3_recount(const orc_params *p, const uint32_t *w, int64_t *n_hb_raw,
                  int64_t *n_coop) {
  int64_t N = (int64_t)p->L * p->L * p->L, hb = 0, co = 0;
  for (int64_t c = 0; c < N; ++c) {
    uint32_t wc = w[c];
    for (int a = 0; a < 6; a += 2)
      if (o3_arm(wc, a) == o3_arm(w[orc3_neighbour(p->L, c, a)], a + 1)) ++hb;
    for (int a = 0; a < 6; ++a)
      for (int b = a + 1; b < 6; ++b)
        if (o3_arm(wc, a) == o3_arm(wc, b)) ++co;
  }
  *n_hb_raw = hb;
  *n_coop = co;
}

int orc3_check_params(const orc_params *p) {
  if (p->L < 2 || p->L > 1024) return ORC_EINVAL;
  if (p->q < 2 || p->q > 8) return ORC_EINVAL;
  if (!(p->kT > 0.0) || !(p->v_iso_init >= 1.0) || !(p->dv_max_frac >= 0.0))
    return ORC_EINVAL;
  if (p->init != ORC_INIT_RANDOM && p->init != ORC_INIT_ORDERED) return ORC_EINVAL;
  if (p->schedule != ORC_SCHED_LAYERED || p->rng_words != 1) return ORC_EINVAL;
  if (p->eta_moves != 0 && p->eta_moves != 1) return ORC_EINVAL;
  if (p->eta_moves && (p->L & 1)) return ORC_EINVAL; /* the cube partition needs L even */
  return ORC_OK;
}

static void o3_start(orc3_state *st, const orc_params *p, uint32_t *w, uint8_t *eta,
                     double V_iso, int64_t sweep) {
  memset(st, 0, sizeof(*st));
  st->p = *p;
  st->N = (int64_t)p->L * p->L * p->L;
  st->w = w;
  st->eta = p->eta_moves ? eta : NULL;
  st->ncube = p->eta_moves ? st->N / 4 : 0;
  st->V_iso = V_iso;
  st->g = (V_iso / (double)st->N < 2.0) ? 1 : 0;
  st->dV_max = p->dv_max_frac * ((double)st->N * p->v_iso_init);
  st->sweep = sweep;
  orc3_threshold_table(p, st->table);
  orc3_eta_table(p, st->eta_table);
  orc3_recount_eta(p, w, st->eta, &st->n_hb_raw, &st->n_coop);
}

/* The initial word of cell c: every sigma 0 (ordered), or sigma_a =
   floor(r q / 2^32) with r word c mod 4 of Philox((c / 4, 0, 0, 16 + a)). */
static uint32_t o3_init_word(const orc_params *p, int64_t c) {
  uint32_t word = 0;
  if (p->init == ORC_INIT_RANDOM)
    for (int a = 0; a < 6; ++a)
      word |= o3_scale(o3_word(p, c, 0, 16u + (uint32_t)a), (uint32_t)p->q) << (4 * a);
  return word;
}

int orc3_init(orc3_state *st, const orc_params *p, uint32_t *w, uint8_t *eta) {
  int rc = orc3_check_params(p);
  if (rc) return rc;
  if (p->eta_moves && !eta) return ORC_EINVAL;
  int64_t N = (int64_t)p->L * p->L * p->L;
  for (int64_t c = 0; c < N; ++c) w[c] = o3_init_word(p, c);
  if (p->eta_moves)
    for (int64_t cube = 0; cube < N / 4; ++cube) eta[cube] = o3_eta_init_cfg(p, cube);
  o3_start(st, p, w, eta, (double)N * p->v_iso_init, 0);
  return ORC_OK;
}

/* Adopt an explicit configuration: sigma words w and, with eta moves, the
   cube configurations eta (each 0..8). */
int orc3_set(orc3_state *st, const orc_params *p, uint32_t *w, uint8_t *eta, double V_iso,
             int64_t sweep) {
  int rc = orc3_check_params(p);
  if (rc) return rc;
  if (p->eta_moves) {
    if (!eta) return ORC_EINVAL;
    int64_t N = (int64_t)p->L * p->L * p->L;
    for (int64_t cube = 0; cube < N / 4; ++cube)
      if (eta[cube] > 8) return ORC_EINVAL;
  }
  o3_start(st, p, w, eta, V_iso, sweep);
  return ORC_OK;
}

/* Volume move (Sec. II.B step 1) with the 2D oracle's readings and the 3D
   cell energy: dV = (2 u1 - 1) dV_max; hard core v' < 1 rejected; gate
   g' = [v' < 2]; dH = N (u(v') - u(v)) + P dV - (g' - g) J_eff N_HB_raw;
   accepted iff u2 < exp(-dH / kT + N ln(V'/V)). */
static double o3_u53(uint32_t hi, uint32_t lo) {
  uint64_t m = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
  return (double)m * (1.0 / 9007199254740992.0);
}

void orc3_volume_move(orc3_state *st) {
  const orc_params *p = &st->p;
  uint32_t r[4];
  o3_philox(p, ORC_CELL_VOLUME, st->sweep, ORC_TAG_VOLUME, r);
  double u1 = o3_u53(r[0], r[1]);
  double u2 = o3_u53(r[2], r[3]);
  double Nd = (double)st->N;
  double dV = (2.0 * u1 - 1.0) * st->dV_max;
  double V_old = st->V_iso;
  double V_new = V_old + dV;
  double v_old = V_old / Nd;
  double v_new = V_new / Nd;
  if (v_new < 1.0) return;
  int32_t g_new = (v_new < 2.0) ? 1 : 0;
  double J_eff = p->J - p->P * p->v_HB;
  double du = orc3_lj_cell_energy(v_new, p->epsilon, p->cutoff) -
              orc3_lj_cell_energy(v_old, p->epsilon, p->cutoff);
  double t1 = Nd * du;
  double t2 = p->P * dV;
  double t3 = ((double)(g_new - st->g) * J_eff) * (double)st->n_hb_raw;
  double dH = (t1 + t2) - t3;
  double arg = -dH / p->kT + Nd * log(V_new / V_old);
  if (u2 < exp(arg)) {
    st->V_iso = V_new;
    st->g = g_new;
    st->acc_volume += 1;
  }
}

/* Permutation number idx (0..719) of the six arms in lexicographic order,
   decoded digit by digit in the factorial number system. */
void orc3_permutation(int idx, int order[6]) {
  int avail[6] = {0, 1, 2, 3, 4, 5};
  int n = 6;
  int fact = 120;
  for (int i = 0; i < 6; ++i) {
    int j = idx / fact;
    idx = idx % fact;
    order[i] = avail[j];
    for (int t = j; t < n - 1; ++t) avail[t] = avail[t + 1];
    --n;
    if (n > 0) fact /= n;
  }
}

void orc3_layer_order(const orc_params *p, int64_t step, int order[6]) {
  uint32_t r[4];
  o3_philox(p, ORC_CELL_LAYERS, step, ORC_TAG_LAYERS, r);
  orc3_permutation((int)o3_scale(r[0], 720u), order);
}

/* Metropolis update of arm a of cell c (Sec. II.C): the proposal is one of
   the q-1 other states; dN_HB compares with arm a^1 of the neighbour in
   direction a, dN_sigma with the five other arms of the cell (Eq. H). */
static void o3_update_arm(orc3_state *st, int64_t c, int a) {
  const orc_params *p = &st->p;
  uint32_t w = o3_word(p, c, st->sweep, 8u + (uint32_t)a);
  uint64_t prod = (uint64_t)w * (uint64_t)(p->q - 1);
  uint32_t k = (uint32_t)(prod >> 32), u = (uint32_t)prod;
  uint32_t wc = st->w[c];
  uint32_t s = o3_arm(wc, a);
  uint32_t sp = (s + 1u + k) % (uint32_t)p->q;
  uint32_t nb = o3_arm(st->w[orc3_neighbour(p->L, c, a)], a ^ 1);
  /* an edge with eta = 0 is no bond whatever its two arms (Eq. H) */
  int dhb = orc3_eta_of(p, st->eta, c, a) ? (sp == nb) - (s == nb) : 0;
  int dc = 0;
  for (int b = 0; b < 6; ++b) {
    if (b == a) continue;
    uint32_t sb = o3_arm(wc, b);
    dc += (sp == sb) - (s == sb);
  }
  if ((uint64_t)u < st->table[st->g][dhb + 1][dc + 5]) {
    st->w[c] = (wc & ~(7u << (4 * a))) | (sp << (4 * a));
    st->n_hb_raw += dhb;
    st->n_coop += dc;
    st->acc_sigma += 1;
  }
}

/* One MC step (Sec. II.B): V_iso, then eta (the cube moves; eta = 1 without
   eta moves), then sigma by six passes over the arm domains in the drawn
   order. */
void orc3_step(orc3_state *st) {
  if (st->p.volume_moves) orc3_volume_move(st);
  if (st->p.eta_moves) orc3_eta_moves(st);
  int order[6];
  orc3_layer_order(&st->p, st->sweep, order);
  for (int pass = 0; pass < 6; ++pass)
    for (int64_t c = 0; c < st->N; ++c) o3_update_arm(st, c, order[pass]);
  st->sweep += 1;
}

/* The initial words of the box x0 <= x < x0 + W, y0 <= y < y0 + H,
   z0 <= z < z0 + D of the L^3 cube w (inside it; nothing else written) and,
   with eta moves, the initial configurations of every checkerboard cube
   with a corner in the box. */
void orc3_init_window(const orc_params *p, uint32_t *w, uint8_t *eta, int32_t x0, int32_t y0,
                      int32_t z0, int32_t W, int32_t H, int32_t D) {
  const int64_t L = p->L;
  for (int64_t z = z0; z < (int64_t)z0 + D; ++z)
    for (int64_t y = y0; y < (int64_t)y0 + H; ++y)
      for (int64_t x = x0; x < (int64_t)x0 + W; ++x) {
        const int64_t c = (z * L + y) * L + x;
        w[c] = o3_init_word(p, c);
        if (p->eta_moves && eta)
          for (int a = 0; a < 6; ++a) {
            int64_t cube;
            int e;
            orc3_edge_of(p->L, c, a, &cube, &e);
            eta[cube] = o3_eta_init_cfg(p, cube);
          }
      }
}

/* K steps over the box alone: step s takes the gate gates[s] (the gate its
   passes use, after its volume move, which the caller's chain provides),
   moves the checkerboard cubes that lie wholly inside the box (with eta
   moves), then runs the six passes in the step's drawn order over the box's
   cells.  A pass moves information by at most one cell along its axis and a
   cube move by one, so a step moves it by at most three along each axis:
   cells more than 3K inside the box are exact (2K without eta moves). */
void orc3_window_run(const orc_params *p, uint32_t *w, uint8_t *eta, int32_t x0, int32_t y0,
                     int32_t z0, int32_t W, int32_t H, int32_t D, int64_t step0, int64_t K,
                     const int32_t *gates) {
  orc3_state st;
  memset(&st, 0, sizeof(st));
  st.p = *p;
  st.N = (int64_t)p->L * p->L * p->L;
  st.w = w;
  st.eta = p->eta_moves ? eta : NULL;
  orc3_threshold_table(p, st.table);
  orc3_eta_table(p, st.eta_table);
  const int64_t L = p->L;
  for (int64_t s = 0; s < K; ++s) {
    st.sweep = step0 + s;
    st.g = gates[s];
    if (st.eta) {
      /* cubes whose corner of smallest coordinates lies in the box with the
         opposite corner inside too (no wrap) */
      for (int64_t cz = z0; cz + 1 < (int64_t)z0 + D; ++cz)
        for (int64_t cy = y0; cy + 1 < (int64_t)y0 + H; ++cy)
          for (int64_t cx = x0; cx + 1 < (int64_t)x0 + W; ++cx) {
            if ((cx & 1) != (cy & 1) || (cx & 1) != (cz & 1)) continue;
            int64_t cube = o3_cube_index(p->L, cx, cy, cz);
            uint32_t r[4];
            o3_philox(p, (uint32_t)cube, st.sweep, O3_TAG_ETA, r);
            uint32_t nw;
            int32_t dhb;
            uint64_t T;
            orc3_eta_probe(p, w, eta, cube, o3_scale(r[0], 8u), st.g, &nw, &dhb, &T);
            if ((uint64_t)r[1] < T) eta[cube] = (uint8_t)nw;
          }
    }
    int order[6];
    orc3_layer_order(p, st.sweep, order);
    for (int pass = 0; pass < 6; ++pass)
      for (int64_t z = z0; z < (int64_t)z0 + D; ++z)
        for (int64_t y = y0; y < (int64_t)y0 + H; ++y)
          for (int64_t x = x0; x < (int64_t)x0 + W; ++x)
            o3_update_arm(&st, (z * L + y) * L + x, order[pass]);
  }
}

/* Observables (Eq. V, Eq. H) and N_q' over all 6N variables. */
void orc3_observables(const orc3_state *st, orc_obs *o) {
  const orc_params *p = &st->p;
  double Nd = (double)st->N;
  int64_t nhb = st->g ? st->n_hb_raw : 0;
  double U = Nd * orc3_lj_cell_energy(st->V_iso / Nd, p->epsilon, p->cutoff);
  double V = st->V_iso + p->v_HB * (double)nhb;
  double H = ((U - p->J * (double)nhb) - p->J_sigma * (double)st->n_coop) + p->P * V;
  memset(o, 0, sizeof(*o));
  o->sweep = st->sweep;
  o->n_hb = nhb;
  o->n_hb_raw = st->n_hb_raw;
  o->n_coop = st->n_coop;
  o->acc_sigma = st->acc_sigma;
  o->acc_volume = st->acc_volume;
  o->V_iso = st->V_iso;
  o->V = V;
  o->U_LJ = U;
  o->H = H;
  o->g = st->g;
  for (int64_t c = 0; c < st->N; ++c)
    for (int a = 0; a < 6; ++a) o->n_state[o3_arm(st->w[c], a)] += 1;
}

int64_t orc3_run(orc3_state *st, int64_t n, int32_t record_every, orc_obs *ring, int64_t cap) {
  int64_t nrec = 0;
  for (int64_t i = 0; i < n; ++i) {
    orc3_step(st);
    if (record_every > 0 && st->sweep % record_every == 0 && ring && nrec < cap)
      orc3_observables(st, &ring[nrec++]);
  }
  return nrec;
}

/* The decision data of arm a of cell c for proposal offset k on an explicit
   configuration: new state and threshold (for the detailed-balance pin). */
void orc3_arm_probe(const orc_params *p, const uint32_t *w, int64_t c, int a, uint32_t k,
                    int32_t g, uint32_t *s_new, uint64_t *T) {
  uint64_t table[2][3][11];
  orc3_threshold_table(p, table);
  uint32_t wc = w[c];
  uint32_t s = o3_arm(wc, a);
  uint32_t sp = (s + 1u + k) % (uint32_t)p->q;
  uint32_t nb = o3_arm(w[orc3_neighbour(p->L, c, a)], a ^ 1);
  int dhb = (sp == nb) - (s == nb);
  int dc = 0;
  for (int b = 0; b < 6; ++b) {
    if (b == a) continue;
    uint32_t sb = o3_arm(wc, b);
    dc += (sp == sb) - (s == sb);
  }
  *s_new = sp;
  *T = table[g][dhb + 1][dc + 5];
}

/* The volume chain alone (no sigma updates) from V_iso with the bonds held
   at n_hb_raw, for the truncated-Gamma pin. */
int64_t orc3_volume_chain(const orc_params *p, double V_iso, int64_t n_hb_raw, int64_t step0,
                          int64_t K, double *V_out) {
  orc3_state st;
  memset(&st, 0, sizeof(st));
  st.p = *p;
  st.N = (int64_t)p->L * p->L * p->L;
  st.V_iso = V_iso;
  st.g = (V_iso / (double)st.N < 2.0) ? 1 : 0;
  st.dV_max = p->dv_max_frac * ((double)st.N * p->v_iso_init);
  st.n_hb_raw = n_hb_raw;
  for (int64_t i = 0; i < K; ++i) {
    st.sweep = step0 + i;
    orc3_volume_move(&st);
    V_out[i] = st.V_iso;
  }
  return st.acc_volume;
}
