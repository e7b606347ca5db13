/*
 * cvf.h -- C ABI of the GB300 (sm_103a) CVF Monte Carlo library.
 *
 * The library runs the Metropolis hot path of the CVF water model of
 * arXiv:2505.05919 on one GPU: the parallel update of the hydrogen-bond
 * indices sigma_ij (Sec. II.C), the counts N_HB and N_sigma of Eq. (H), and
 * the isobaric update of the global volume V_iso (Sec. II.B, step 1), on a
 * periodic 2D square lattice with one molecule and four bonding indices per
 * cell (q states each).  One Monte Carlo step ("sweep") is: one volume move,
 * then every sigma once (Sec. II.B order V_iso -> eta -> sigma; eta is
 * identically 1 in 2D because a cell has exactly four neighbours).
 *
 * Conventions shared by every entry point
 *   - Every call returns an int status: CVF_OK (0) or one of the CVF_E*
 *     codes below.  cvf_last_error() gives a text for the calling thread's
 *     last failure.
 *   - Units are reduced (Table 1): energies in eps (5.5 kJ/mol), lengths in
 *     r0 (2.9 A), volumes in v0 = r0^3.  cvf_params_physical converts
 *     (T [K], P [MPa]).
 *   - Lattice layout: cell c = y*L + x (x fastest), one uint16 word per cell
 *     holding sigma of arm a in bits [4a, 4a+3) -- one nibble per arm, bits
 *     3, 7, 11 and 15 zero.  Arms
 *     0..3 = left, right, front, back; arm 0 points to +x, arm 1 to -x, arm 2
 *     to +y, arm 3 to -y (the paper's worked example of Sec. II.C: arm 0 of
 *     cell c pairs with arm 1 of cell c+1).  A bond joins arm a of a cell
 *     with arm a^1 of its neighbour in direction a.
 *   - Streams: every handle enqueues its GPU work on the cudaStream_t given
 *     at creation (passed as void*; NULL = the legacy default stream).  Calls
 *     that return host data synchronise that stream; the others are
 *     asynchronous.
 *   - Ownership: host buffers are always the caller's.  Device memory the
 *     library allocates is freed by the matching destroy call.  A device
 *     buffer the caller passes in stays the caller's and must outlive the
 *     handle.
 *   - Thread safety: a handle must not be used from two threads at once.
 */
#ifndef CVF_H
#define CVF_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CVF_OK 0
#define CVF_EINVAL 1    /* invalid argument or parameter */
#define CVF_ENOMEM 2    /* device or host allocation failed */
#define CVF_ECUDA 3     /* a CUDA runtime call failed */
#define CVF_ETIMEOUT 4  /* a bounded device-side wait gave up */
#define CVF_EBUSY 5     /* the handle has work that conflicts with the call */
#define CVF_EOVERFLOW 6 /* the observable ring overwrote unread records */
#define CVF_EBOUNDS 7   /* a debug build's device-side index check failed */

#define CVF_INIT_RANDOM 0
#define CVF_INIT_ORDERED 1
#define CVF_SCHED_CHECKERBOARD 0
#define CVF_SCHED_LAYERED 1

/* Model and run parameters (reduced units).  Sec. II.A names: J and J_sigma
 * are the covalent and cooperative hydrogen-bond energies of Eq. (H), v_HB
 * the volume per bond of Eq. (V), epsilon and cutoff the Lennard-Jones
 * energy and range (Table 1), kT and P the thermodynamic state. */
typedef struct cvf_params {
  int32_t L;            /* lattice side, even, 2 <= L <= 65534 */
  int32_t q;            /* states per bonding index, 2 <= q <= 8 (q = 6, Sec. II.A) */
  double epsilon;       /* LJ energy scale (1 = eps; 0 switches U_LJ off) */
  double cutoff;        /* LJ cutoff in r0 (6, Sec. II.A) */
  double J;             /* covalent HB energy (2.0 = J/(4 eps) 0.5, Table 1) */
  double J_sigma;       /* cooperative energy (0.32 = J_sigma/(4 eps) 0.08) */
  double v_HB;          /* volume per HB in v0 (0.6, Sec. II.A) */
  double kT;            /* temperature, kT/eps > 0 */
  double P;             /* pressure, P v0/eps */
  double v_iso_init;    /* initial V_iso / N in v0 (>= 1; default 2^(1/3)) */
  double dv_max_frac;   /* volume step: |dV| <= dv_max_frac * N v_iso_init */
  uint64_t seed;        /* Philox4x32-10 key (low word, high word) */
  int32_t init;         /* CVF_INIT_RANDOM or CVF_INIT_ORDERED (all sigma 0) */
  int32_t schedule;     /* CVF_SCHED_CHECKERBOARD (default) or CVF_SCHED_LAYERED */
  int32_t volume_moves; /* 1: isobaric volume move each step; 0: fixed V_iso */
  int32_t rng_words;    /* 1: one 32-bit word per update (default); 2: two */
  int32_t eta_moves;    /* cubic lattice only: 1 = the eta update of App. A
                           (default of cvf3_params_physical; needs L even),
                           0 = eta identically 1.  Must be 0 on the square
                           lattice, where eta is identically 1 */
  int32_t pad;          /* zero */
} cvf_params;

/* Observables after a completed step (Eq. V and Eq. H). */
typedef struct cvf_obs {
  int64_t sweep;      /* completed MC steps */
  int64_t n_hb;       /* N_HB = g * N_HB_raw (gas cells form no bonds) */
  int64_t n_hb_raw;   /* pairs with sigma_ij == sigma_ji */
  int64_t n_coop;     /* N_sigma: equal pairs inside the cells */
  int64_t acc_sigma;  /* accepted sigma moves since creation/set_state */
  int64_t acc_volume; /* accepted volume moves since creation/set_state */
  double V_iso;       /* isotropic volume, v0 */
  double V;           /* V = V_iso + v_HB N_HB (Eq. V) */
  double U_LJ;        /* Lennard-Jones energy, eps */
  double H;           /* H = U_LJ - J N_HB - J_sigma N_sigma + P V (Eq. H) */
  int32_t g;          /* gate: 1 liquid-like (V_iso/N < 2 v0), 0 gas-like */
  int32_t status;     /* 0; 1 if a bounded device-side wait gave up (the
                         call then returns CVF_ETIMEOUT); 0x100 + site if a
                         debug build's index check at `site` failed
                         (CVF_EBOUNDS) */
  int64_t n_state[8]; /* N_q': sigma variables in state q' (q' >= q: 0);
                         the order parameter is M = max N_q' / (4N),
                         Eq. (correlation) */
} cvf_obs;

typedef struct cvf_handle cvf_handle;
typedef struct cvf_batch cvf_batch;

/* Text of the calling thread's last error ("" when none).  The pointer is
 * valid until the next failing call on the same thread. */
const char *cvf_last_error(void);

/* Fills *out with the Table 1 parameters (L = 64, q = 6, epsilon = 1,
 * cutoff = 6, J = 2, J_sigma = 0.32, v_HB = 0.6, v_iso_init = 2^(1/3),
 * dv_max_frac = 0.01, seed 1, random init, checkerboard, volume moves on,
 * one RNG word per update) at T = 300 K, P = 0.1 MPa. */
int cvf_params_default(cvf_params *out);

/* Table 1 parameters at the physical state point (T_kelvin, P_MPa):
 * kT/eps = T R / 5.5 kJ/mol, P v0/eps = P r0^3 N_A / 5.5 kJ/mol.
 * CVF_EINVAL if T_kelvin <= 0 or out is NULL. */
int cvf_params_physical(double T_kelvin, double P_MPa, cvf_params *out);

/* The 42 Metropolis thresholds of the parameters (Sec. II.C with Eq. H),
 * laid out [g][dN_HB + 1][dN_sigma + 3] for g in {0,1}, dN_HB in {-1,0,1},
 * dN_sigma in {-3..3}: T = 2^32 when dH = -g J_eff dN_HB - J_sigma dN_sigma
 * <= 0, else floor(exp(-dH/kT) 2^32), J_eff = J - P v_HB.  A move is
 * accepted when its 32-bit draw u satisfies u < T.  Host only. */
int cvf_threshold_table(const cvf_params *p, uint64_t out[42]);

/* Creates a lattice handle and initialises it on the device (random init
 * from Philox((c, 0, 0, 2), seed) or all sigma = 0), with V_iso = N
 * v_iso_init, N_HB_raw and N_sigma counted, sweep = 0.
 *   stream     cudaStream_t as void* (NULL: legacy default stream).
 *   dev_state  NULL: the library allocates the lattice.  Otherwise a device
 *              buffer of 2*L*L uint16 words (the lattice and its double
 *              buffer), 16-byte aligned, owned by the caller.
 *   out        receives the handle.
 * CVF_EINVAL for invalid parameters, CVF_ENOMEM/CVF_ECUDA on device
 * failure (nothing is leaked). */
int cvf_create(const cvf_params *p, void *stream, void *dev_state,
               cvf_handle **out);

/* Enqueues n_sweeps MC steps (volume move, then the checkerboard -- or
 * layered -- sigma sweep).  When record_every > 0 the observables after
 * every step whose count is a multiple of record_every are appended to the
 * device ring (capacity 65536 records, read with cvf_drain_series).  The
 * steps run as CUDA graphs; the call returns without waiting.
 * CVF_EINVAL if n_sweeps < 0 or record_every < 0. */
int cvf_sweep(cvf_handle *h, int64_t n_sweeps, int32_t record_every);

/* Observables after the last completed step; synchronises the stream.
 * N_sigma and N_q' are counted from the lattice by this call.  Returns
 * CVF_ETIMEOUT (with *out filled) if a bounded wait in a sweep gave up. */
int cvf_observables(cvf_handle *h, cvf_obs *out);

/* Moves the unread ring records (oldest first) into host[0..cap) and sets
 * *n to their number; synchronises the stream.  Returns CVF_EOVERFLOW (with
 * the newest records still delivered) when records were overwritten since
 * the last drain. */
int cvf_drain_series(cvf_handle *h, cvf_obs *host, int64_t cap, int64_t *n);

/* Copies the lattice (L*L words, layout above) to host; synchronises.
 * CVF_EINVAL if n != L*L. */
int cvf_get_state(cvf_handle *h, uint16_t *host, size_t n);

/* Copies the rectangle of cells x0 <= x < x0 + W, y0 <= y < y0 + H (inside
 * the lattice, no wrap) to host[0 .. W*H), row by row (host[(y - y0) W +
 * (x - x0)] = word of cell x + L y); synchronises.  For reading parts of
 * lattices too large to copy whole.  CVF_EINVAL if the rectangle is empty
 * or leaves the lattice. */
int cvf_get_window(cvf_handle *h, int32_t x0, int32_t y0, int32_t W, int32_t H,
                   uint16_t *host);

/* Replaces the lattice by host[0..n) (n = L*L), sets V_iso and the step
 * counter, recounts N_HB_raw and N_sigma, and clears the acceptance
 * counters and the ring.  The words are uploaded into the state pair's free
 * buffer and validated there on the device before they replace the lattice
 * (arms < q, bits 3, 7, 11, 15 zero): CVF_EINVAL otherwise, naming the
 * first invalid word, with nothing changed.
 * V_iso must be >= N (the hard core).  Synchronises. */
int cvf_set_state(cvf_handle *h, const uint16_t *host, size_t n, double V_iso,
                  int64_t sweep);

/* Recounts N_HB_raw and N_sigma from the current lattice with a separate
 * reduction kernel (independent of the counts the sweep maintains);
 * synchronises. */
int cvf_recount(cvf_handle *h, int64_t *n_hb_raw, int64_t *n_sigma);

/* Device address of the current lattice (L*L words), valid until the next
 * call that enqueues work on the handle. */
int cvf_state_device_ptr(cvf_handle *h, void **dev_ptr);

/* Tile shape of the checkerboard sweep: config 0 = 64 rows x 64 words (128
 * cells), 1 = 32 x 32, 2 = 16 x 32, 3 = the whole lattice resident in the
 * shared memory of one thread-block cluster (8 CTAs hold rows, a ninth
 * decides the volume moves ahead) for many steps per launch (16 <= L <=
 * 256, L a multiple of 8; rows = L/8 per CTA); 4, 5, 6 = the tiles of 0, 1,
 * 2 swept by one persistent cooperative launch per call in which a tile of
 * step s + 1 waits only for the tiles around it to finish step s (a
 * wavefront; the volume moves decided ahead by one block; L a multiple of 8
 * and at least 3 x 3 tiles); -1 = automatic (chosen at creation: the
 * resident form for small lattices, else the largest tile shape whose tiles
 * fill every resident block, swept as a wavefront from L = 256 up).  The result does not depend on the config;
 * set_tiles waits for the stream.  CVF_EINVAL for other values, or a config
 * that does not apply to the lattice. */
int cvf_set_tiles(cvf_handle *h, int32_t config);
int cvf_get_tiles(cvf_handle *h, int32_t *config, int32_t *rows,
                  int32_t *words);

/* Waits for the handle's stream, frees what the library allocated. */
int cvf_destroy(cvf_handle *h);

/* Allocation-free sweep.  The paper has no counterpart: this entry point is
 * for callers that cannot let a library call cudaMalloc -- applications that
 * own all device memory through their own pool, or that must not allocate
 * once running because an allocation can synchronise the device or fail
 * under memory pressure in the middle of a run.  It advances a caller-owned
 * lattice by n_sweeps MC steps (checkerboard schedule) and allocates nothing:
 * the control block, counters, thresholds, FP64 parameters and up to 256
 * recorded observable sets live in a fixed 64 KB device array that the
 * library defines at file scope (every GPU that loads the library holds it
 * until the process exits).
 *   dev_state    device buffer of 2*L*L uint16 words (16-byte aligned): the
 *                lattice is read from half (sweep & 1) and left in half
 *                ((sweep + n_sweeps) & 1); the other half is overwritten.
 *   V_iso, sweep the volume and the step count the run continues from
 *                (acceptance counters start at 0 for the call).
 *   record_every observables after every step whose count is a multiple of
 *                it are copied to host_series[0..series_cap) (at most 256 per
 *                call, else CVF_EINVAL); *n_series receives their number.
 *   host_obs     receives the observables after the last step.
 * dev_state must hold valid cells for q (guard bits clear, every nibble < q);
 * the call checks this on the device and returns CVF_EINVAL after the run
 * when it does not hold (the lattice is then swept anyway and its contents
 * are meaningless).  After the stream synchronises the call returns the
 * lattice's status as cvf_observables does: CVF_ETIMEOUT when a bounded
 * device wait gave up, CVF_EBOUNDS when an index check of a debug build
 * failed; *n_series and host_obs are filled in either case.  A launch that
 * fails ends the call with CVF_ECUDA.
 * The call synchronises `stream`.  Every call looks up the array's device
 * address on the current device (cudaGetSymbolAddress), so the address stays
 * right across a device reset.  Every call on a device uses the same array
 * and clears what must start at zero, so calls whose GPU work overlaps (other
 * threads, other streams) race with each other: serialise them. */
int cvf_sweep_noalloc(const cvf_params *p, void *dev_state, double V_iso,
                      int64_t sweep, int64_t n_sweeps, int32_t record_every,
                      cvf_obs *host_series, int64_t series_cap,
                      int64_t *n_series, cvf_obs *host_obs, void *stream);

/* ------------------------------------------------------------------------
 * Batched replicas: many independent lattices (their own L, q, T, P, seed,
 * init) advanced by one persistent, cooperative, graph-captured launch.
 * Every replica computes exactly what cvf_create + cvf_sweep compute for it
 * alone (same steps, same counter-based draws).  Replicas use the
 * checkerboard schedule and share rng_words.  Replica ids are slot numbers
 * 0 .. n_slots-1; a removed slot is reused by a later add.
 * ------------------------------------------------------------------------ */

/* Creates a batch holding n replicas with parameters params[0..n) (n may be
 * 0), each initialised as by cvf_create; ids are 0..n-1.  Work is enqueued on
 * stream (cudaStream_t as void*).  CVF_EINVAL for invalid parameters, a
 * layered schedule or differing rng_words; CVF_ENOMEM when device memory
 * runs out (nothing leaked). */
int cvf_batch_create(const cvf_params *params, int32_t n, void *stream,
                     cvf_batch **out);

/* Adds one replica and returns its id: allocates its state pair, control
 * block, tables and a 1024-record observable ring from the batch's
 * stream-ordered memory pool and enqueues its initialisation on the stream,
 * behind any launch in flight.  Does not wait for the GPU: the parameters
 * travel as kernel arguments, so p may be reused on return.  CVF_ENOMEM
 * when the device has no room for it (nothing leaked). */
int cvf_batch_add(cvf_batch *b, const cvf_params *p, int32_t *replica);

/* Frees a replica, stream-ordered: its memory goes back to the batch's pool
 * once the work already enqueued on the stream has run (no wait here).  Its
 * id becomes free at once; the replica's results must be read before. */
int cvf_batch_remove(cvf_batch *b, int32_t replica);

/* Number of slots (live or free) and of live replicas. */
int cvf_batch_size(cvf_batch *b, int32_t *n_slots, int32_t *n_live);

/* Advances replica i by sweeps[i] MC steps, i = 0..n-1 with n the slot count
 * (0 for free slots and for replicas to leave alone), in one persistent
 * launch; returns without waiting for it (the launch description goes
 * through one of two pinned staging slots, so a call waits at most for the
 * copy enqueued two calls before).  At most 64 distinct nonzero step counts
 * and 2^31-1 steps per replica per call.  A bounded device-side wait that
 * gives up is reported by the next call that reads results (CVF_ETIMEOUT). */
int cvf_batch_sweep(cvf_batch *b, const int64_t *sweeps, int32_t n);

/* Waits for the batch's stream; CVF_ETIMEOUT if the last launch gave up. */
int cvf_batch_sync(cvf_batch *b);

/* Observables / lattice (L*L words, layout above) of one replica; both
 * synchronise the stream. */
int cvf_batch_observables(cvf_batch *b, int32_t replica, cvf_obs *out);

/* Observables of n replicas (ids replicas[0..n), out[0..n)), each as
 * cvf_batch_observables returns it, with one synchronisation of the stream.
 * CVF_EINVAL for an id that is not a live replica (nothing read). */
int cvf_batch_observables_many(cvf_batch *b, const int32_t *replicas,
                               int32_t n, cvf_obs *out);

/* The same read in two halves, so the host need not wait for work enqueued
 * after it.  _enqueue computes the n replicas' observables at the current
 * point of the stream (after the sweeps already enqueued, before any later
 * call's work), copies them and the launch error word into pinned staging,
 * and returns a ticket without waiting.  _collect waits for that point of
 * the stream only (an event), then fills out[0..n) (n as enqueued) or
 * returns the error of the sweeps before it (CVF_ETIMEOUT / CVF_EBOUNDS as
 * cvf_batch_sync).  Four tickets stay valid at a time: the fifth enqueue
 * reuses the first one's staging (CVF_EINVAL when it is then collected). */
int cvf_batch_observables_enqueue(cvf_batch *b, const int32_t *replicas,
                                  int32_t n, int64_t *ticket);
int cvf_batch_observables_collect(cvf_batch *b, int64_t ticket, cvf_obs *out,
                                  int32_t n);
int cvf_batch_get_state(cvf_batch *b, int32_t replica, uint16_t *host,
                        size_t n);

/* Kernel configuration of the batched sweep: config c >= 0 selects a tile
 * of rows x 32-bit words and a block size from a fixed list of twelve
 * (cvf_batch_tile_config, cvf_batch_config_threads): configs 0..3 are the
 * tiles 64x64, 32x32, 32x16, 16x16 (rows x words) with 256-thread blocks,
 * configs 4..7 the same tiles with 128-thread blocks and 8..11 with
 * 512-thread blocks, so a thread updates 2 rows words / threads cells per
 * MC step independently of the tile.  -1
 * (the default) chooses per call: the largest 256-thread tile whose count
 * over the replicas the call advances is at least the kernel's co-resident
 * blocks; else the smallest tile, with 512-thread blocks (config 11) when
 * its count is below a quarter of the blocks and 256-thread blocks (config
 * 3) otherwise.  cvf_batch_get_tiles returns the setting and the
 * configuration the last call used (-1 before any call). */
int cvf_batch_set_tiles(cvf_batch *b, int32_t config);
int cvf_batch_get_tiles(cvf_batch *b, int32_t *config, int32_t *last_used);
int cvf_batch_tile_config(int32_t config, int32_t *rows, int32_t *words);
int cvf_batch_config_threads(int32_t config, int32_t *threads);

/* Device memory the batch's pool has mapped (reserved) and of that what
 * live replicas and the descriptor array hold (used); reserved - used is
 * free for later adds but not for other allocations. */
int cvf_batch_memory(cvf_batch *b, uint64_t *reserved, uint64_t *used);

/* Waits for the stream and frees every replica, the pool and the batch. */
int cvf_batch_destroy(cvf_batch *b);

/* ------------------------------------------------------------------------
 * The paper's own 3D model: a periodic cubic lattice of N = L^3 cells with
 * six bonding indices per cell (Sec. II.A: six nearest neighbours), updated
 * by the layered partition of Sec. II.C -- the six arm domains one after the
 * other, in an order drawn every MC step -- with up to C(6,2) = 15
 * cooperative pairs per cell in Eq. (H), and (eta_moves = 1) the eta update
 * of App. A: every molecule keeps exactly four allowed bonds.
 *   - eta: the checkerboard cubes are the unit cells whose corner of
 *     smallest coordinates (cx, cy, cz) has all three coordinates even
 *     (colour 0) or all odd (colour 1); each molecule is a corner of one cube
 *     of each colour and each edge lies in exactly one cube, so the L^3/4
 *     cubes (L even) partition the 3N edges.  A cube's configuration is the
 *     set of its edges with eta = 0: one of the nine perfect matchings of
 *     the cube graph, numbered 0..8 in increasing order of their 12-bit edge
 *     mask (edge e runs along axis e / 4 from the (e % 4)-th corner, in
 *     increasing corner number, whose offset along that axis is 0; corner j
 *     sits at offset (j & 1, (j >> 1) & 1, (j >> 2) & 1)).  Cube index:
 *     colour (L/2)^3 + (Z (L/2) + Y) (L/2) + X for the cube at (2X + colour,
 *     2Y + colour, 2Z + colour).  Step 2 of every MC step moves each cube by
 *     Metropolis: configuration (c + 1 + k) mod 9, k = floor(r0 8 / 2^32),
 *     accepted iff r1 < T, T = 2^32 min(1, exp(g J_eff dN_HB / kT)) floored,
 *     r = Philox((cube, step, 5)); random init takes configuration
 *     floor(r0 9 / 2^32) of Philox((cube, 0, 0, 6)), ordered init 0.  A bond
 *     counts in N_HB (and in the sigma moves) only on an edge with eta = 1.
 *   - Layout: cell c = x + L (y + L z), one uint32 word per cell holding
 *     sigma of arm a in bits [4a, 4a+3) -- one nibble per arm, bits 4a+3 and
 *     24..31 zero in every word the calls below exchange.  (Inside the
 *     library bit 4a+3 holds the eta of arm a's edge: a caller reading the
 *     device buffer directly masks it off with 0x777777.)  Arms 0..5 =
 *     left, right, front, back, top, bottom point to +x, -x, +y, -y, +z, -z
 *     (Sec. II.C's coalescing example and Table S1: arm 0 of cell c pairs
 *     with arm 1 of cell c+1, arm 4 of cell (1,0,0) with arm 5 of (1,0,1)).
 *   - One MC step: the volume move (Sec. II.B, with the cubic-lattice LJ
 *     energy u(v) = 2 eps [v^-4 S12 - v^-2 S6], r = v^(1/3)), then six
 *     passes, pass i updating arm order[i] of every cell; order is the
 *     permutation number floor(w 720 / 2^32) (lexicographic) of the six arms,
 *     w word 0 of Philox((2^32-2, step, 4)).
 *   - Draws: the update of arm a of cell c in step s uses word c mod 4 of
 *     Philox((c / 4, s, 8 + a), seed): w (q-1) = k 2^32 + u gives the
 *     proposal sigma' = (sigma + 1 + k) mod q and the acceptance draw u;
 *     random init sigma_a(c) = floor(w q / 2^32), w word c mod 4 of
 *     Philox((c / 4, 0, 16 + a)).
 *   - Parameters: cvf_params with L the cube side (2 <= L <= 1024), schedule
 *     CVF_SCHED_LAYERED and rng_words 1 (other values: CVF_EINVAL);
 *     v_iso_init defaults to 2^(1/2) (the pair minimum r = 2^(1/6) r0);
 *     eta_moves 1 needs an even L.
 *   - Observables: cvf_obs as above with N_HB <= 2N with eta moves (3N
 *     without), N_sigma <= 15N and the order parameter M = max N_q' / (6N).
 *     n_hb_raw counts the equal arm pairs on edges with eta = 1.
 * Streams, ownership, errors and thread safety as for cvf_handle.
 * ------------------------------------------------------------------------ */
typedef struct cvf3_handle cvf3_handle;

/* Table 1 parameters at (T_kelvin, P_MPa) for the cubic lattice: as
 * cvf_params_physical with L = 16, v_iso_init = 2^(1/2), the layered
 * schedule, one RNG word per update and the eta moves of App. A. */
int cvf3_params_physical(double T_kelvin, double P_MPa, cvf_params *out);

/* The 66 thresholds [g][dN_HB + 1][dN_sigma + 5] (dN_sigma in -5..5, the
 * five other arms of the cell): T = 2^32 when dH = -g J_eff dN_HB -
 * J_sigma dN_sigma <= 0, else floor(exp(-dH/kT) 2^32).  Host only. */
int cvf3_threshold_table(const cvf_params *p, uint64_t out[66]);

/* Creates a cubic lattice on the device (random or ordered init), V_iso =
 * N v_iso_init, counts N_HB_raw and N_sigma, sweep = 0.
 *   dev_state  NULL: the library allocates the lattice; otherwise a device
 *              buffer of L^3 uint32 words, 16-byte aligned, owned by the
 *              caller (the passes update it in place). */
int cvf3_create(const cvf_params *p, void *stream, void *dev_state,
                cvf3_handle **out);

/* Enqueues n_sweeps MC steps (graph-captured; returns without waiting);
 * record_every as for cvf_sweep (ring of 65536 records). */
int cvf3_sweep(cvf3_handle *h, int64_t n_sweeps, int32_t record_every);

/* Observables after the last completed step (N_q' counted from the lattice
 * by this call); synchronises.  N_HB_raw and N_sigma are the counts the
 * passes maintain incrementally. */
int cvf3_observables(cvf3_handle *h, cvf_obs *out);

/* As cvf_drain_series. */
int cvf3_drain_series(cvf3_handle *h, cvf_obs *host, int64_t cap, int64_t *n);

/* Copies / replaces the lattice (n = L^3 words, layout above).  set_state
 * validates every word on the host (arms < q, other bits zero), sets V_iso
 * (>= N) and the step counter, recounts, clears the acceptance counters and
 * the ring.  Both synchronise. */
int cvf3_get_state(cvf3_handle *h, uint32_t *host, size_t n);

/* Copies the box x0 <= x < x0 + W, y0 <= y < y0 + H, z0 <= z < z0 + D
 * (inside the cube, no wrap) to host[0 .. W*H*D), x fastest
 * (host[((z - z0) H + (y - y0)) W + (x - x0)] = word of cell x + L (y + L z));
 * synchronises.  CVF_EINVAL if the box is empty or leaves the cube. */
int cvf3_get_window(cvf3_handle *h, int32_t x0, int32_t y0, int32_t z0, int32_t W,
                    int32_t H, int32_t D, uint32_t *host);
int cvf3_set_state(cvf3_handle *h, const uint32_t *host, size_t n,
                   double V_iso, int64_t sweep);

/* The cube configurations (App. A), n = L^3 / 4 bytes, each 0..8, in the
 * cube order above.  get copies them to the host; set replaces them (every
 * value checked on the host, CVF_EINVAL otherwise, and without eta moves),
 * recounts N_HB_raw and prepares the next volume move.  Checkpoint and
 * resume: cvf3_set_state, then cvf3_set_eta.  Both synchronise. */
int cvf3_get_eta(cvf3_handle *h, uint8_t *host, size_t n);
int cvf3_set_eta(cvf3_handle *h, const uint8_t *host, size_t n);

/* Recounts N_HB_raw (bonds on allowed edges) and N_sigma with a separate
 * reduction; synchronises. */
int cvf3_recount(cvf3_handle *h, int64_t *n_hb_raw, int64_t *n_sigma);

/* Device address of the lattice (L^3 words; bit 4a+3 of a word holds the
 * eta of arm a's edge, see the layout above). */
int cvf3_state_device_ptr(cvf3_handle *h, void **dev_ptr);

/* Form of the sweep: mode 1 keeps the cube in the shared memory of one
 * thread-block cluster for all the steps of a call (L a multiple of 8,
 * 16 <= L <= 64; 16 CTAs where L is a multiple of 16 from 32 up and the GPU
 * can place such a cluster, else 8; the z-planes split among the CTAs; with
 * eta moves each CTA moves the cubes whose lower plane it holds), 0 runs the
 * step as launches over the cube in global memory, -1 chooses.  The results
 * do not depend on the form; the call waits for the stream.  CVF_EINVAL for
 * mode 1 where it does not apply.  The automatic choice (-1, the default at
 * creation) takes the resident form up to L = 24, and at L = 32 with a
 * 16-CTA cluster. */
int cvf3_set_resident(cvf3_handle *h, int32_t mode);
int cvf3_get_resident(cvf3_handle *h, int32_t *resident);

/* Waits for the handle's stream, frees what the library allocated. */
int cvf3_destroy(cvf3_handle *h);

/* ------------------------------------------------------------------------
 * Measurement aid: the byte roofline of the sweep's working set.
 *
 * The sweep's algorithmic traffic is 2 B read + 2 B written per cell and MC
 * step (1 B per sigma update).  A 4096^2 lattice (32 MB) stays in the L2
 * cache across steps, so the byte roofline that bounds it is the L2 copy
 * bandwidth, which no vendor figure states; timing this copy on two buffers
 * that together fit in L2 measures it (and on buffers far larger than L2,
 * the DRAM copy bandwidth).
 *
 * cvf_copy_probe: enqueue one copy of `bytes` from device buffer `src` to
 * device buffer `dst` on `stream` (a cudaStream_t; NULL = legacy default
 * stream) with 16-byte loads and stores.  Both pointers and `bytes` must be
 * multiples of 16 and the buffers must not overlap; the caller owns both.
 * Asynchronous: returns after the launch.  CVF_EINVAL for a NULL or
 * misaligned argument, CVF_ECUDA if the launch fails.
 * ------------------------------------------------------------------------ */
int cvf_copy_probe(void *dst, const void *src, size_t bytes, void *stream);

/* cvf_philox_probe: enqueue the random-number work of one checkerboard step
 * and nothing else: for every cell c < n_cells one Philox4x32-10 block with
 * counter (c, step_lo, step_hi, 0) and key `seed` (the draws of cell c in
 * MC step `step` with one word per update; Salmon et al., SC'11), computed
 * by the same
 * device function as the sweep kernels.  The 4 n_cells words are XOR-folded
 * into *dev_out (atomic XOR, so the caller zeroes it first; caller-owned
 * device memory, 4-byte aligned), which keeps every draw live and lets a
 * test check the words against another Philox implementation.  Timed with
 * events, 4 n_cells / time is the most sigma updates per second a sweep
 * that draws one block per cell can reach on this GPU: the measured ceiling
 * beside which the sweep's rate is reported.  Asynchronous; CVF_EINVAL for
 * a NULL or misaligned output or a negative step. */
int cvf_philox_probe(uint64_t seed, uint32_t n_cells, int64_t step, uint32_t *dev_out,
                     void *stream);

/* 1 if this library was built with device-side index checks (CVF_DEBUG:
 * every kernel checks its shared- and global-memory indices and the TMA
 * alignment rule, records the first failing site in the lattice's status
 * word, skips the access, and the calls that read results return
 * CVF_EBOUNDS), 0 for the release build.  Host only. */
int cvf_debug_checks(void);

/* ------------------------------------------------------------------------
 * Failure detection without a fault.
 *
 * Every device-side wait of the library is bounded: a tile of the persistent
 * batched sweep (cvf_batch_sweep) that waits for its replica's previous step
 * polls a progress word with acquire loads, sleeping about 128 min(d, 8)^2 ns
 * between polls when the word is d short of its target, and gives up after
 * about half a second of such sleep, after which the launch ends and the next
 * call that reads results returns CVF_ETIMEOUT with the context intact.
 *
 * cvf_wait_probe: run that same wait alone: one device thread polls the
 * 4-byte-aligned device word `flag` until it is >= `target`, with a budget of
 * `polls` 128-ns sleep quanta (1 <= polls <= 2^22; a poll d short of the
 * target uses min(d, 8)^2 of them, so one per poll when the flag is one
 * short).  Synchronises `stream` (a cudaStream_t; NULL =
 * legacy default stream).  Returns CVF_OK when the value was seen,
 * CVF_ETIMEOUT when the wait gave up (a flag that nothing sets), CVF_EINVAL
 * for a NULL or misaligned flag or `polls` out of range, CVF_ECUDA if a CUDA
 * call failed.  The caller owns `flag`; the library writes nothing to it.
 * ------------------------------------------------------------------------ */
int cvf_wait_probe(const uint32_t *flag, uint32_t target, uint32_t polls, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CVF_H */
