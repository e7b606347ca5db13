/*
 * cvf_oracle.c -- plain, slow, single-threaded CPU oracle of the CVF 2D
 * Metropolis hot path (arXiv:2505.05919).
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the CPU legs
 * of bench.py (cpu_baseline, --impl reference) may load, call or run this
 * file.  The product library never does; the two share no code, header,
 * table or constant generator.
 *
 * What it computes, and where each step comes from:
 *   - the model: Sec. II.A (Eq. V, Eq. vi, Eq. H, Table 1), restricted to the
 *     2D periodic square lattice with four bonding indices per cell and one
 *     molecule per cell (the bulk case, every n_i = 1);
 *   - the MC step order V_iso -> eta -> sigma: Sec. II.B (eta is identically 1
 *     in 2D because a cell has exactly four neighbours, so its update is a
 *     no-op);
 *   - the Metropolis update of the sigma_ij: Sec. II.C, with the enthalpy
 *     change of Eq. H and J_eff = J - P v_HB (Fig. 1 caption);
 *   - random numbers: counter-based Philox4x32-10 (Salmon, Moraes, Dror,
 *     Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), replacing
 *     the pre-generated cuRAND arrays of App. C.
 * Where the paper is silent the readings used here are listed in the design
 * notes (proposal set, schedule, volume-move proposal and acceptance, LJ
 * prefactor and cutoff, 2D units, RNG word mapping); each is restated in the
 * comment of the function that applies it.
 *
 * Arithmetic: uint32/uint64 for the RNG and the thresholds, int64 for the
 * counters, IEEE double (compile with -ffp-contract=off) for the volume and
 * the enthalpy.  Compile: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "cvf_oracle.h"

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (SC'11): a 4x32-bit counter, a 2x32-bit key, ten rounds.  */
/* One round multiplies counter words 0 and 2 by the two Philox constants,  */
/* keeps both halves of each 64-bit product, and mixes the high halves with */
/* the other two counter words and the round key.  The key is advanced by   */
/* the two Weyl constants between rounds.                                   */
/* ------------------------------------------------------------------------ */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_WEYL_0 0x9E3779B9u
#define ORC_WEYL_1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t prod0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)x0;
    uint64_t prod1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)x2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t y0 = hi1 ^ x1 ^ k0;
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x3 ^ k1;
    uint32_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    k0 += ORC_WEYL_0;
    k1 += ORC_WEYL_1;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The four words drawn for (counter word 0, MC step, stream tag). */
static void orc_draw(const orc_params *p, uint32_t word0, int64_t step,
                     uint32_t tag, uint32_t out[4]) {
  uint32_t ctr[4] = {word0, (uint32_t)((uint64_t)step & 0xFFFFFFFFu),
                     (uint32_t)((uint64_t)step >> 32), tag};
  uint32_t key[2] = {(uint32_t)(p->seed & 0xFFFFFFFFu),
                     (uint32_t)(p->seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* floor(w * n / 2^32): an integer in [0, n) from one 32-bit word. */
static uint32_t orc_scale(uint32_t w, uint32_t n) {
  return (uint32_t)(((uint64_t)w * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Lattice geometry (2D reading of Sec. II.C): cell c = y*L + x, periodic,  */
/* x fastest (the cell <-> (x,y,z) column of the label-equivalence table).  */
/* Arms 0..3 = left, right, front, back, the 2D subset of the paper's order. */
/* The worked layout example of Sec. II.C (arm 0 of cells 0..15 reads arm 1 */
/* of cells 1..16) puts the "left" partner of cell c at c+1, i.e. arm 0     */
/* points to +x and arm 1 to -x; by the same rule arm 2 points to +y and    */
/* arm 3 to -y.  A bond of arm a pairs with arm a^1 of the neighbour in     */
/* direction a.  Packed word: sigma of arm a in bits [4a, 4a+3).            */
/* ------------------------------------------------------------------------ */
static int64_t orc_neighbour(int32_t L, int64_t c, int arm) {
  int64_t x = c % L, y = c / L;
  switch (arm) {
    case 0: x = (x + 1) % L; break;
    case 1: x = (x + L - 1) % L; break;
    case 2: y = (y + 1) % L; break;
    default: y = (y + L - 1) % L; break;
  }
  return y * L + x;
}

/* Bond partner of (cell, arm): the neighbour cell in direction arm and the
   arm of that cell the bond pairs with. */
void orc_bond_partner(int32_t L, int64_t c, int arm, int64_t *c_out,
                      int *arm_out) {
  *c_out = orc_neighbour(L, c, arm);
  *arm_out = arm ^ 1;
}

/* Cell word: sigma of arm a in bits [4a, 4a+3), one nibble per arm; bits
   4a+3 are zero. */
static uint32_t orc_arm(uint16_t word, int arm) {
  return ((uint32_t)word >> (4 * arm)) & 7u;
}

/* ------------------------------------------------------------------------ */
/* Lennard-Jones energy per cell (Sec. II.A, Table 1).  Reading: the 2D     */
/* lattice is a monolayer of thickness r0, so v_iso = r^2 r0 and, in units   */
/* of r0 and v0 = r0^3, the squared distance of a pair separated by lattice  */
/* vector d is |d|^2 v_iso.  A pair contributes 4 eps [(r0/dist)^12 -        */
/* (r0/dist)^6] when dist < cutoff (strict).  Every cell sees the same       */
/* infinite-lattice neighbourhood, so U_LJ = N u(v_iso) with                 */
/*   u(v) = 1/2 sum_{d != 0, |d|^2 v < cutoff^2} 4 eps [(1/(|d|^2 v))^6 -    */
/*          (1/(|d|^2 v))^3],                                                */
/* the half giving each cell its share of every pair.  The sum is taken     */
/* pair by pair, shell by shell (the m lattice vectors of one |d|^2 give     */
/* equal terms), in increasing |d|^2.  v >= 1 is the hard core.              */
/* ------------------------------------------------------------------------ */
#define ORC_MAX_SHELLS 4096
static int orc_shells(double cutoff, int64_t d2s[], int64_t mult[]) {
  /* Integer enumeration of the lattice vectors that can lie inside the
     cutoff at the hard-core density v = 1, grouped by |d|^2. */
  int R = (int)ceil(cutoff) + 1;
  int n = 0;
  for (int64_t d2 = 1; d2 <= (int64_t)R * R * 2; ++d2) {
    int64_t m = 0;
    for (int i = -R; i <= R; ++i)
      for (int j = -R; j <= R; ++j)
        if ((int64_t)i * i + (int64_t)j * j == d2) ++m;
    if (m > 0 && (double)d2 < cutoff * cutoff) {
      if (n >= ORC_MAX_SHELLS) return -1;
      d2s[n] = d2;
      mult[n] = m;
      ++n;
    }
  }
  return n;
}

double orc_lj_cell_energy(double v_iso, double epsilon, double cutoff) {
  /* the shell list depends on the cutoff only */
  static int64_t d2s[ORC_MAX_SHELLS], mult[ORC_MAX_SHELLS];
  static double last_cutoff = -1.0;
  static int n = 0;
  if (cutoff != last_cutoff) {
    n = orc_shells(cutoff, d2s, mult);
    if (n < 0) n = 0;
    last_cutoff = cutoff;
  }
  double rc2 = cutoff * cutoff;
  double sum = 0.0;
  for (int s = 0; s < n; ++s) {
    double dist2 = (double)d2s[s] * v_iso; /* (r / r0)^2 of this shell's pairs */
    if (!(dist2 < rc2)) break;            /* shells ascend: the rest lie outside */
    double y = 1.0 / dist2;               /* (r0 / r)^2 */
    double y3 = y * y * y;                /* (r0 / r)^6 */
    double y6 = y3 * y3;                  /* (r0 / r)^12 */
    double pair = (4.0 * epsilon) * (y6 - y3);
    sum += (double)mult[s] * pair;
  }
  return 0.5 * sum;
}

int orc_shell_table(double cutoff, int64_t *d2s, int64_t *mult, int cap) {
  static int64_t a[ORC_MAX_SHELLS], b[ORC_MAX_SHELLS];
  int n = orc_shells(cutoff, a, b);
  if (n < 0 || n > cap) return -1;
  for (int i = 0; i < n; ++i) { d2s[i] = a[i]; mult[i] = b[i]; }
  return n;
}

/* ------------------------------------------------------------------------ */
/* Metropolis threshold table (Sec. II.C with Eq. H).  Changing one sigma   */
/* changes N_HB_raw by dhb in {-1,0,1} and N_sigma by dc in {-3..3}; the    */
/* enthalpy changes by dH = -g J_eff dhb - J_sigma dc, where the P v_HB N_HB */
/* part of P V is folded into J_eff = J - P v_HB and the gas/liquid gate g   */
/* multiplies only the N_HB term (Eq. H).  A move is accepted when a 32-bit  */
/* draw u satisfies u < T, T = 2^32 when dH <= 0 and floor(exp(-dH/kT) 2^32)  */
/* otherwise: min(1, exp(-dH/kT)) resolved to 2^-32.                        */
/* ------------------------------------------------------------------------ */
void orc_threshold_table(const orc_params *p, uint64_t out[2][3][7]) {
  double J_eff = p->J - p->P * p->v_HB;
  for (int g = 0; g < 2; ++g)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 7; ++j) {
        int dhb = i - 1, dc = j - 3;
        double dH = -((double)g * J_eff) * (double)dhb - p->J_sigma * (double)dc;
        uint64_t T;
        if (dH <= 0.0)
          T = (uint64_t)1 << 32;
        else
          T = (uint64_t)(exp(-dH / p->kT) * 4294967296.0);
        out[g][i][j] = T;
      }
}

/* ------------------------------------------------------------------------ */
/* Counters (Eq. H): N_HB_raw = number of bonded pairs sigma_ij = sigma_ji  */
/* over all nearest-neighbour pairs (each bond once, via arms 0 and 2 of     */
/* every cell, the +x and +y bonds); N_coop = N_sigma = number of equal pairs of sigma    */
/* within each cell, summed over cells (at most C(4,2) = 6 per cell).  The   */
/* gated count is N_HB = g N_HB_raw.                                         */
/* ------------------------------------------------------------------------ */
void orc_recount(const orc_params *p, const uint16_t *w, int64_t *n_hb_raw,
                 int64_t *n_coop) {
  int32_t L = p->L;
  int64_t N = (int64_t)L * L, hb = 0, coop = 0;
  for (int64_t c = 0; c < N; ++c) {
    uint16_t wc = w[c];
    if (orc_arm(wc, 0) == orc_arm(w[orc_neighbour(L, c, 0)], 1)) ++hb;
    if (orc_arm(wc, 2) == orc_arm(w[orc_neighbour(L, c, 2)], 3)) ++hb;
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b)
        if (orc_arm(wc, a) == orc_arm(wc, b)) ++coop;
  }
  *n_hb_raw = hb;
  *n_coop = coop;
}

/* ------------------------------------------------------------------------ */
/* Validation of the parameters this oracle supports.                       */
/* ------------------------------------------------------------------------ */
int orc_check_params(const orc_params *p) {
  if (p->L < 2 || (p->L & 1) || p->L > 65535) return ORC_EINVAL;
  if (p->q < 2 || p->q > 8) return ORC_EINVAL;
  if (!(p->kT > 0.0) || !(p->cutoff > 0.0)) return ORC_EINVAL;
  if (!(p->v_iso_init >= 1.0)) return ORC_EINVAL;
  if (!(p->dv_max_frac >= 0.0)) return ORC_EINVAL;
  if (p->init != ORC_INIT_RANDOM && p->init != ORC_INIT_ORDERED)
    return ORC_EINVAL;
  if (p->schedule != ORC_SCHED_CHECKERBOARD && p->schedule != ORC_SCHED_LAYERED)
    return ORC_EINVAL;
  if (p->rng_words != 1 && p->rng_words != 2) return ORC_EINVAL;
  /* a square-lattice cell has exactly four neighbours: every eta is 1 */
  if (p->eta_moves != 0) return ORC_EINVAL;
  return ORC_OK;
}

static void orc_set_volume(orc_state *st, double V_iso) {
  st->V_iso = V_iso;
  double v = V_iso / (double)st->N;
  st->g = (v < 2.0) ? 1 : 0;
}

/* Initial configuration (App. B: the host builds the initial sigma).  Random
   init: sigma_a(c) = floor(w_a q / 2^32) with w = Philox((c, 0, 0, 2), seed).
   Ordered init: every sigma = 0, so every bond is formed and every in-cell
   pair is equal.  V_iso starts at N v_iso_init (the paper gives no initial
   volume; the default per-cell value is the pair-LJ minimum 2^(1/3) v0). */
/* The initial word of cell c: every sigma 0 (ordered), or sigma_a =
   floor(r_a q / 2^32) with r = Philox((c, 0, 0, 2)) (random). */
static uint16_t orc_init_word(const orc_params *p, int64_t c) {
  uint16_t word = 0;
  if (p->init == ORC_INIT_RANDOM) {
    uint32_t r[4];
    orc_draw(p, (uint32_t)c, 0, ORC_TAG_INIT, r);
    for (int a = 0; a < 4; ++a)
      word |= (uint16_t)(orc_scale(r[a], (uint32_t)p->q) << (4 * a));
  }
  return word;
}

int orc_init(orc_state *st, const orc_params *p, uint16_t *w) {
  int rc = orc_check_params(p);
  if (rc) return rc;
  memset(st, 0, sizeof(*st));
  st->p = *p;
  st->N = (int64_t)p->L * p->L;
  st->w = w;
  for (int64_t c = 0; c < st->N; ++c) w[c] = orc_init_word(p, c);
  orc_set_volume(st, (double)st->N * p->v_iso_init);
  st->dV_max = p->dv_max_frac * ((double)st->N * p->v_iso_init);
  orc_threshold_table(p, st->table);
  orc_recount(p, w, &st->n_hb_raw, &st->n_coop);
  return ORC_OK;
}

/* Adopt an explicit configuration (checkpoint restore); counters recounted. */
int orc_set(orc_state *st, const orc_params *p, uint16_t *w, double V_iso,
            int64_t sweep) {
  int rc = orc_check_params(p);
  if (rc) return rc;
  memset(st, 0, sizeof(*st));
  st->p = *p;
  st->N = (int64_t)p->L * p->L;
  st->w = w;
  for (int64_t c = 0; c < st->N; ++c)
    for (int a = 0; a < 4; ++a)
      if (orc_arm(w[c], a) >= (uint32_t)p->q || (w[c] & 0x8888u)) return ORC_EINVAL;
  orc_set_volume(st, V_iso);
  st->dV_max = p->dv_max_frac * ((double)st->N * p->v_iso_init);
  st->sweep = sweep;
  orc_threshold_table(p, st->table);
  orc_recount(p, w, &st->n_hb_raw, &st->n_coop);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Volume move (Sec. II.B, step 1).  The paper states only that V_iso moves */
/* by +-O(V_iso/100) with a Metropolis test involving exp(-P dV_iso / kT).   */
/* Reading applied here: dV = (2 u1 - 1) dV_max with dV_max = dv_max_frac    */
/* times the initial V_iso (fixed, so the proposal is symmetric); v_iso' < v0 */
/* is the hard core and is rejected; the enthalpy change includes the LJ     */
/* term, P dV_iso and the change of gate g' = [v_iso' < 2 v0] on the bonded  */
/* pairs, and the acceptance carries the isobaric Jacobian N ln(V'/V):       */
/*   accept iff u2 < exp(-dH/kT + N ln(V'/V)).                               */
/* u1, u2 are 53-bit uniforms from Philox((2^32-1, step, 3)).                */
/* ------------------------------------------------------------------------ */
static double orc_u53(uint32_t hi, uint32_t lo) {
  uint64_t m = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
  return (double)m * (1.0 / 9007199254740992.0);
}

void orc_volume_move(orc_state *st) {
  const orc_params *p = &st->p;
  uint32_t r[4];
  orc_draw(p, ORC_CELL_VOLUME, st->sweep, ORC_TAG_VOLUME, r);
  double u1 = orc_u53(r[0], r[1]);
  double u2 = orc_u53(r[2], r[3]);
  double Nd = (double)st->N;
  double dV = (2.0 * u1 - 1.0) * st->dV_max;
  double V_old = st->V_iso;
  double V_new = V_old + dV;
  double v_old = V_old / Nd;
  double v_new = V_new / Nd;
  if (v_new < 1.0) return; /* hard core: r < r0 is forbidden */
  int32_t g_new = (v_new < 2.0) ? 1 : 0;
  double J_eff = p->J - p->P * p->v_HB;
  double du = orc_lj_cell_energy(v_new, p->epsilon, p->cutoff) -
              orc_lj_cell_energy(v_old, p->epsilon, p->cutoff);
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

/* ------------------------------------------------------------------------ */
/* One Metropolis update of arm `arm` of cell c (Sec. II.C).  Proposal: a    */
/* new value uniform over the q-1 other states, sigma' = (sigma + 1 + k) mod */
/* q with k = floor(p (q-1) / 2^32) (the "(sigma + rnd) % q" idiom of        */
/* Sec. II.D).  The change of N_HB_raw compares with arm a^1 of the          */
/* neighbour in direction a; the change of N_sigma compares with the other   */
/* three arms of the same cell as they are now.  Words: rng_words = 2 takes  */
/* the acceptance draw from tag 0 and the proposal word from tag 1;          */
/* rng_words = 1 takes both from the tag-0 word w, via w (q-1) = k 2^32 + u. */
/* ------------------------------------------------------------------------ */
static void orc_words(const orc_state *st, int64_t c, uint32_t acc[4],
                      uint32_t kk[4]) {
  const orc_params *p = &st->p;
  uint32_t u[4], pw[4];
  orc_draw(p, (uint32_t)c, st->sweep, ORC_TAG_ACCEPT, u);
  if (p->rng_words == 2) {
    orc_draw(p, (uint32_t)c, st->sweep, ORC_TAG_PROPOSE, pw);
    for (int a = 0; a < 4; ++a) {
      acc[a] = u[a];
      kk[a] = orc_scale(pw[a], (uint32_t)(p->q - 1));
    }
  } else {
    for (int a = 0; a < 4; ++a) {
      uint64_t prod = (uint64_t)u[a] * (uint64_t)(p->q - 1);
      kk[a] = (uint32_t)(prod >> 32);
      acc[a] = (uint32_t)prod;
    }
  }
}

/* The decision data of one arm update: proposed value, changes of the two
   counters and the threshold it is compared against. */
static void orc_arm_decision(const orc_params *p, const uint64_t table[2][3][7],
                             int32_t g, const uint16_t *w, int64_t c, int arm,
                             uint32_t k, uint32_t *s_new, int *dhb_out,
                             int *dc_out, uint64_t *T_out) {
  uint16_t wc = w[c];
  uint32_t s = orc_arm(wc, arm);
  uint32_t sp = (s + 1u + k) % (uint32_t)p->q;
  uint32_t nb = orc_arm(w[orc_neighbour(p->L, c, arm)], arm ^ 1);
  int dhb = (sp == nb) - (s == nb);
  int dc = 0;
  for (int b = 0; b < 4; ++b) {
    if (b == arm) continue;
    uint32_t sb = orc_arm(wc, b);
    dc += (sp == sb) - (s == sb);
  }
  *s_new = sp;
  *dhb_out = dhb;
  *dc_out = dc;
  *T_out = table[g][dhb + 1][dc + 3];
}

static void orc_update_arm(orc_state *st, int64_t c, int arm, uint32_t acc,
                           uint32_t k) {
  uint32_t sp;
  int dhb, dc;
  uint64_t T;
  orc_arm_decision(&st->p, st->table, st->g, st->w, c, arm, k, &sp, &dhb, &dc,
                   &T);
  if ((uint64_t)acc < T) {
    uint16_t wc = st->w[c];
    wc = (uint16_t)((wc & ~(7u << (4 * arm))) | (sp << (4 * arm)));
    st->w[c] = wc;
    st->n_hb_raw += dhb;
    st->n_coop += dc;
    st->acc_sigma += 1;
  }
}

/* Checkerboard schedule (reading of Sec. II.C for 2D): colour (x+y)&1,
   colour 0 first; a colour's cells interact only through the other colour,
   so each colour is one domain of simultaneous updates.  Within a cell the
   four arms are updated in the order 0..3, each seeing the earlier ones. */
static void orc_sweep_checkerboard(orc_state *st) {
  int32_t L = st->p.L;
  for (int colour = 0; colour < 2; ++colour)
    for (int64_t y = 0; y < L; ++y)
      for (int64_t x = 0; x < L; ++x) {
        if (((x + y) & 1) != colour) continue;
        int64_t c = y * L + x;
        uint32_t acc[4], kk[4];
        orc_words(st, c, acc, kk);
        for (int a = 0; a < 4; ++a) orc_update_arm(st, c, a, acc[a], kk[a]);
      }
}

/* Layered schedule (Sec. II.C as printed): one arm domain at a time, in an
   order drawn per step (Fisher-Yates with words from Philox((2^32-2, step,
   4))); a domain holds the same arm of every cell, which interact only with
   other domains, so all of them move together.  Each update uses the same
   per-cell words as the checkerboard schedule. */
void orc_layer_order(const orc_params *p, int64_t step, int order[4]) {
  uint32_t r[4];
  orc_draw(p, ORC_CELL_LAYERS, step, ORC_TAG_LAYERS, r);
  for (int a = 0; a < 4; ++a) order[a] = a;
  for (int i = 3; i >= 1; --i) {
    int j = (int)orc_scale(r[3 - i], (uint32_t)(i + 1));
    int t = order[i];
    order[i] = order[j];
    order[j] = t;
  }
}

static void orc_sweep_layered(orc_state *st) {
  int order[4];
  orc_layer_order(&st->p, st->sweep, order);
  for (int pass = 0; pass < 4; ++pass) {
    int a = order[pass];
    for (int64_t c = 0; c < st->N; ++c) {
      uint32_t acc[4], kk[4];
      orc_words(st, c, acc, kk);
      orc_update_arm(st, c, a, acc[a], kk[a]);
    }
  }
}

/* One MC step (Sec. II.B): V_iso, then eta (a no-op in 2D), then sigma. */
void orc_step(orc_state *st) {
  if (st->p.volume_moves) orc_volume_move(st);
  if (st->p.schedule == ORC_SCHED_LAYERED)
    orc_sweep_layered(st);
  else
    orc_sweep_checkerboard(st);
  st->sweep += 1;
}

/* Observables (Eq. V and Eq. H): N_HB = g N_HB_raw, V = V_iso + v_HB N_HB,
   U_LJ = N u(v_iso), H = U_LJ - J N_HB - J_sigma N_sigma + P V; and N_q', the
   number of sigma variables in each state q' (Eq. correlation, the counts
   the order parameter M is the maximum of). */
void orc_observables(const orc_state *st, orc_obs *o) {
  const orc_params *p = &st->p;
  double Nd = (double)st->N;
  int64_t nhb = st->g ? st->n_hb_raw : 0;
  double U = Nd * orc_lj_cell_energy(st->V_iso / Nd, p->epsilon, p->cutoff);
  double V = st->V_iso + p->v_HB * (double)nhb;
  double H = ((U - p->J * (double)nhb) - p->J_sigma * (double)st->n_coop) +
             p->P * V;
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
    for (int a = 0; a < 4; ++a) o->n_state[orc_arm(st->w[c], a)] += 1;
}

/* n steps; after every step whose new count is a multiple of record_every
   (when record_every > 0) the observables are appended to ring[0..cap). */
int64_t orc_run(orc_state *st, int64_t n, int32_t record_every, orc_obs *ring,
                int64_t cap) {
  int64_t nrec = 0;
  for (int64_t i = 0; i < n; ++i) {
    orc_step(st);
    if (record_every > 0 && st->sweep % record_every == 0 && nrec < cap && ring)
      orc_observables(st, &ring[nrec++]);
  }
  return nrec;
}

/* ------------------------------------------------------------------------ */
/* Probes used by the pins.                                                  */
/* ------------------------------------------------------------------------ */

/* Decision data of one arm update on an explicit configuration, for the
   single-variable detailed-balance check. */
void orc_arm_probe(const orc_params *p, const uint16_t *w, int64_t c, int arm,
                   uint32_t k, int32_t g, uint32_t *s_new, int32_t *dhb,
                   int32_t *dc, uint64_t *T) {
  uint64_t table[2][3][7];
  int a, b;
  orc_threshold_table(p, table);
  orc_arm_decision(p, table, g, w, c, arm, k, s_new, &a, &b, T);
  *dhb = a;
  *dc = b;
}

/* Batched form over many configurations of one lattice (n configurations
   of L*L words each), every cell and arm and every proposal offset k in
   [0, q-1): out arrays are indexed [cfg][cell][arm][k]. */
void orc_arm_probe_all(const orc_params *p, const uint16_t *cfgs, int64_t n,
                       int32_t g, uint32_t *s_new, uint64_t *T) {
  uint64_t table[2][3][7];
  orc_threshold_table(p, table);
  int64_t N = (int64_t)p->L * p->L;
  int q1 = p->q - 1;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t c = 0; c < N; ++c)
      for (int a = 0; a < 4; ++a)
        for (int k = 0; k < q1; ++k) {
          int dhb, dc;
          int64_t o = ((i * N + c) * 4 + a) * q1 + k;
          orc_arm_decision(p, table, g, cfgs + i * N, c, a, (uint32_t)k,
                           &s_new[o], &dhb, &dc, &T[o]);
        }
}

/* Steps restricted to a rectangular window of a full L x L configuration:
   only cells (x mod L, y mod L) with x0 <= x < x0+W and y0 <= y < y0+H are
   updated (a window may run across the periodic edges; W, H <= L), the rest
   stay frozen, and the gate of each step is taken from gates[].  After K
   steps every window cell farther than 2K cells from the window edge equals
   the full-lattice result, because a checkerboard step moves information by
   at most two cells.  The volume chain is not run here. */
void orc_window_run(const orc_params *p, uint16_t *w, int32_t x0, int32_t y0,
                    int32_t W, int32_t H, int64_t step0, int64_t K,
                    const int32_t *gates) {
  orc_state st;
  memset(&st, 0, sizeof(st));
  st.p = *p;
  st.N = (int64_t)p->L * p->L;
  st.w = w;
  orc_threshold_table(p, st.table);
  for (int64_t s = 0; s < K; ++s) {
    st.sweep = step0 + s;
    st.g = gates[s];
    for (int colour = 0; colour < 2; ++colour)
      for (int64_t yy = y0; yy < (int64_t)y0 + H; ++yy)
        for (int64_t xx = x0; xx < (int64_t)x0 + W; ++xx) {
          int64_t x = xx % p->L, y = yy % p->L;
          if (((x + y) & 1) != colour) continue;
          int64_t c = y * p->L + x;
          uint32_t acc[4], kk[4];
          orc_words(&st, c, acc, kk);
          for (int a = 0; a < 4; ++a) orc_update_arm(&st, c, a, acc[a], kk[a]);
        }
  }
}

/* The initial words of the cells (x mod L, y mod L), x0 <= x < x0 + W,
   y0 <= y < y0 + H, of the L x L lattice w (W, H <= L; nothing else is
   written), so that a window of a lattice too large to initialise whole can
   be started and run by orc_window_run. */
void orc_init_window(const orc_params *p, uint16_t *w, int32_t x0, int32_t y0,
                     int32_t W, int32_t H) {
  for (int64_t yy = y0; yy < (int64_t)y0 + H; ++yy)
    for (int64_t xx = x0; xx < (int64_t)x0 + W; ++xx) {
      int64_t c = (yy % p->L) * p->L + xx % p->L;
      w[c] = orc_init_word(p, c);
    }
}

/* The V_iso chain alone for K steps from (V_iso, step0), valid while no
   proposal changes the gate (then the acceptance does not involve the
   sigma).  Writes V_iso and the gate after each step's move (the gate each
   step's sweep uses).  Returns the number of steps done before the first
   proposal that would change the gate (K when there is none). */
int64_t orc_volume_chain(const orc_params *p, double V_iso, int64_t step0,
                         int64_t K, double *V_out, int32_t *g_out,
                         int64_t *acc_out) {
  orc_state st;
  memset(&st, 0, sizeof(st));
  st.p = *p;
  st.N = (int64_t)p->L * p->L;
  st.dV_max = p->dv_max_frac * ((double)st.N * p->v_iso_init);
  orc_set_volume(&st, V_iso);
  for (int64_t s = 0; s < K; ++s) {
    st.sweep = step0 + s;
    if (p->volume_moves) {
      uint32_t r[4];
      orc_draw(p, ORC_CELL_VOLUME, st.sweep, ORC_TAG_VOLUME, r);
      double dV = (2.0 * orc_u53(r[0], r[1]) - 1.0) * st.dV_max;
      double v_new = (st.V_iso + dV) / (double)st.N;
      if (v_new >= 1.0 && ((v_new < 2.0) ? 1 : 0) != st.g) return s;
      orc_volume_move(&st);
    }
    V_out[s] = st.V_iso;
    g_out[s] = st.g;
  }
  if (acc_out) *acc_out = st.acc_volume;
  return K;
}
