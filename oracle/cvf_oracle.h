/*
 * cvf_oracle.h -- interface of the CPU oracle (test infrastructure only; see
 * cvf_oracle.c).  This header belongs to the oracle alone: the CUDA library
 * has its own, independent definitions.
 */
#ifndef CVF_ORACLE_H
#define CVF_ORACLE_H
#include <stdint.h>

#define ORC_OK 0
#define ORC_EINVAL 1

#define ORC_INIT_RANDOM 0
#define ORC_INIT_ORDERED 1
#define ORC_SCHED_CHECKERBOARD 0
#define ORC_SCHED_LAYERED 1

/* Philox counter word 3 (stream tag) and the reserved counter word 0 values */
#define ORC_TAG_ACCEPT 0u
#define ORC_TAG_PROPOSE 1u
#define ORC_TAG_INIT 2u
#define ORC_TAG_VOLUME 3u
#define ORC_TAG_LAYERS 4u
#define ORC_CELL_VOLUME 0xFFFFFFFFu
#define ORC_CELL_LAYERS 0xFFFFFFFEu

/* Parameters in reduced units: energies in eps, lengths in r0, volumes in
   v0 = r0^3 (Table 1). */
typedef struct {
  int32_t L, q;
  double epsilon, cutoff;
  double J, J_sigma, v_HB;
  double kT, P;
  double v_iso_init, dv_max_frac;
  uint64_t seed;
  int32_t init, schedule, volume_moves, rng_words;
  int32_t eta_moves; /* 3D only: 1 = the eta update of App. A, 0 = eta = 1 */
  int32_t pad;
} orc_params;

typedef struct {
  int64_t sweep, n_hb, n_hb_raw, n_coop, acc_sigma, acc_volume;
  double V_iso, V, U_LJ, H;
  int32_t g, pad;
  int64_t n_state[8]; /* number of sigma variables in each state q' */
} orc_obs;

typedef struct {
  orc_params p;
  int64_t N;
  uint16_t *w;
  double V_iso, dV_max;
  int64_t sweep, n_hb_raw, n_coop, acc_sigma, acc_volume;
  int32_t g, pad;
  uint64_t table[2][3][7];
} orc_state;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);
double orc_lj_cell_energy(double v_iso, double epsilon, double cutoff);
int orc_shell_table(double cutoff, int64_t *d2s, int64_t *mult, int cap);
void orc_threshold_table(const orc_params *p, uint64_t out[2][3][7]);
void orc_recount(const orc_params *p, const uint16_t *w, int64_t *n_hb_raw,
                 int64_t *n_coop);
int orc_check_params(const orc_params *p);
void orc_bond_partner(int32_t L, int64_t c, int arm, int64_t *c_out,
                      int *arm_out);
int orc_init(orc_state *st, const orc_params *p, uint16_t *w);
int orc_set(orc_state *st, const orc_params *p, uint16_t *w, double V_iso,
            int64_t sweep);
void orc_volume_move(orc_state *st);
void orc_step(orc_state *st);
void orc_observables(const orc_state *st, orc_obs *o);
int64_t orc_run(orc_state *st, int64_t n, int32_t record_every, orc_obs *ring,
                int64_t cap);
void orc_layer_order(const orc_params *p, int64_t step, int order[4]);
void orc_arm_probe(const orc_params *p, const uint16_t *w, int64_t c, int arm,
                   uint32_t k, int32_t g, uint32_t *s_new, int32_t *dhb,
                   int32_t *dc, uint64_t *T);
void orc_arm_probe_all(const orc_params *p, const uint16_t *cfgs, int64_t n,
                       int32_t g, uint32_t *s_new, uint64_t *T);
void orc_init_window(const orc_params *p, uint16_t *w, int32_t x0, int32_t y0,
                     int32_t W, int32_t H);
void orc_window_run(const orc_params *p, uint16_t *w, int32_t x0, int32_t y0,
                    int32_t W, int32_t H, int64_t step0, int64_t K,
                    const int32_t *gates);
int64_t orc_volume_chain(const orc_params *p, double V_iso, int64_t step0,
                         int64_t K, double *V_out, int32_t *g_out,
                         int64_t *acc_out);
/* ---- 3D variant (cvf_oracle3.c): cubic lattice, six arms per cell, one
   nibble each (sigma in its low 3 bits) in one uint32 word, layered
   schedule. ---- */
typedef struct {
  orc_params p;
  int64_t N;
  uint32_t *w;
  double V_iso, dV_max;
  int64_t sweep, n_hb_raw, n_coop, acc_sigma, acc_volume;
  int32_t g, pad;
  uint64_t table[2][3][11];
  /* eta (App. A): one configuration number 0..8 per checkerboard cube
     (N / 4 cubes), the move thresholds [g][dN_HB + 4] and the number of
     accepted cube moves; eta == NULL when eta_moves is 0 (eta = 1) */
  uint8_t *eta;
  int64_t ncube, acc_eta;
  uint64_t eta_table[2][9];
} orc3_state;

int64_t orc3_neighbour(int32_t L, int64_t c, int arm);
int orc3_shell_table(double cutoff, int64_t *d2s, int64_t *mult, int cap);
double orc3_lj_cell_energy(double v_iso, double epsilon, double cutoff);
void orc3_threshold_table(const orc_params *p, uint64_t out[2][3][11]);
void orc3_recount(const orc_params *p, const uint32_t *w, int64_t *n_hb_raw,
                  int64_t *n_coop);
int orc3_check_params(const orc_params *p);
int orc3_init(orc3_state *st, const orc_params *p, uint32_t *w, uint8_t *eta);
int orc3_set(orc3_state *st, const orc_params *p, uint32_t *w, uint8_t *eta,
             double V_iso, int64_t sweep);
int orc3_matchings(uint16_t out[9]);
void orc3_cube_corner_cells(int32_t L, int64_t cube, int64_t cells[8]);
void orc3_edge_of(int32_t L, int64_t c, int a, int64_t *cube, int *e);
int orc3_eta_of(const orc_params *p, const uint8_t *eta, int64_t c, int a);
void orc3_eta_table(const orc_params *p, uint64_t out[2][9]);
void orc3_eta_moves(orc3_state *st);
void orc3_eta_probe(const orc_params *p, const uint32_t *w, const uint8_t *eta,
                    int64_t cube, uint32_t k, int32_t g, uint32_t *cfg_new,
                    int32_t *dhb, uint64_t *T);
void orc3_recount_eta(const orc_params *p, const uint32_t *w, const uint8_t *eta,
                      int64_t *n_hb_raw, int64_t *n_coop);
void orc3_volume_move(orc3_state *st);
void orc3_permutation(int idx, int order[6]);
void orc3_layer_order(const orc_params *p, int64_t step, int order[6]);
void orc3_step(orc3_state *st);
void orc3_observables(const orc3_state *st, orc_obs *o);
int64_t orc3_run(orc3_state *st, int64_t n, int32_t record_every, orc_obs *ring,
                 int64_t cap);
void orc3_arm_probe(const orc_params *p, const uint32_t *w, int64_t c, int a,
                    uint32_t k, int32_t g, uint32_t *s_new, uint64_t *T);
void orc3_init_window(const orc_params *p, uint32_t *w, uint8_t *eta, int32_t x0, int32_t y0,
                      int32_t z0, int32_t W, int32_t H, int32_t D);
void orc3_window_run(const orc_params *p, uint32_t *w, uint8_t *eta, int32_t x0, int32_t y0,
                     int32_t z0, int32_t W, int32_t H, int32_t D, int64_t step0, int64_t K,
                     const int32_t *gates);
int64_t orc3_volume_chain(const orc_params *p, double V_iso, int64_t n_hb_raw,
                          int64_t step0, int64_t K, double *V_out);
#endif
