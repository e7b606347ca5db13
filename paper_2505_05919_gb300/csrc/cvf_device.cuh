// cvf_device.cuh -- device building blocks of the CVF Metropolis path
// (arXiv:2505.05919): counter-based Philox4x32-10 words and the draws of a
// cell, cell-word helpers, the FP64 isobaric volume move, the end of a step
// and block reductions.  Included by the kernel translation units only.
#pragma once
#include <cstdint>
#include <type_traits>

#include "cvf.h"

namespace cvf {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11).  The counter is (c, step_lo, step_hi,
// tag); the key is the 64-bit seed.  Ten rounds; the round keys are the seed
// words advanced by the Weyl constants and are computed once on the host.
// ---------------------------------------------------------------------------
constexpr uint32_t kPhiloxMul0 = 0xD2511F53u;
constexpr uint32_t kPhiloxMul1 = 0xCD9E8D57u;
constexpr uint32_t kWeyl0 = 0x9E3779B9u;
constexpr uint32_t kWeyl1 = 0xBB67AE85u;

constexpr uint32_t kTagAccept = 0u;   // acceptance words (and proposals, 1 word/update)
constexpr uint32_t kTagPropose = 1u;  // proposal words (2 words/update)
constexpr uint32_t kTagInit = 2u;     // random initial sigma
constexpr uint32_t kTagVolume = 3u;   // volume move
constexpr uint32_t kTagLayers = 4u;   // layered-schedule arm order
constexpr uint32_t kCellVolume = 0xFFFFFFFFu;
constexpr uint32_t kCellLayers = 0xFFFFFFFEu;

// Round r's two key words side by side (k[r].x for word 0, k[r].y for word
// 1), so a copy in shared memory is read with one 8-byte load per round.
struct RoundKeys {
  uint2 k[10];
};

inline RoundKeys make_round_keys(uint64_t seed) {
  RoundKeys K;
  uint32_t a = (uint32_t)(seed & 0xFFFFFFFFu), b = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    K.k[r] = make_uint2(a, b);
    a += kWeyl0;
    b += kWeyl1;
  }
  return K;
}

struct Words4 {
  uint32_t x, y, z, w;
};

// Ten Philox rounds on (x0, x1, x2, x3): counter words 0 and 2 are multiplied
// by the Philox constants; the high halves are mixed with words 1, 3 and the
// round key, the low halves become the new words 1 and 3.
__device__ __forceinline__ Words4 philox(uint32_t x0, uint32_t x1, uint32_t x2,
                                         uint32_t x3, const RoundKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t m0 = (uint64_t)x0 * kPhiloxMul0;
    const uint64_t m1 = (uint64_t)x2 * kPhiloxMul1;
    const uint2 kr = K.k[r];
    const uint32_t y0 = (uint32_t)(m1 >> 32) ^ x1 ^ kr.x;
    const uint32_t y2 = (uint32_t)(m0 >> 32) ^ x3 ^ kr.y;
    x1 = (uint32_t)m1;
    x3 = (uint32_t)m0;
    x0 = y0;
    x2 = y2;
  }
  return Words4{x0, x1, x2, x3};
}

// The same ten rounds for counters (c, step_lo, step_hi, tag) whose last
// three words are shared by every cell of a step.  Rounds 0-2 multiply step_hi
// and then the round-0 output word A = hi(step_hi M1) ^ step_lo ^ k0.x, which
// are the same for every cell; their products and the key words they are
// XORed with fold into four words per (step, tag), computed once:
//   b = tag ^ k0.y,  c = lo(step_hi M1) ^ k1.x,  d = hi(A M0) ^ k1.y,
//   e = lo(A M0) ^ k2.y.
// philox_cell(c, philox_step(step_lo, step_hi, tag, K), K) equals
// philox(c, step_lo, step_hi, tag, K) bit for bit (XORs reassociated only),
// with 18 widening multiplies and 19 XORs per cell instead of 20 and 20.
struct PhiloxStep {
  uint32_t b, c, d, e;
};

__host__ __device__ inline PhiloxStep philox_step(uint32_t step_lo, uint32_t step_hi, uint32_t tag,
                                                  const RoundKeys& K) {
  const uint64_t m1 = (uint64_t)step_hi * kPhiloxMul1;
  const uint32_t A = (uint32_t)(m1 >> 32) ^ step_lo ^ K.k[0].x;
  const uint64_t mA = (uint64_t)A * kPhiloxMul0;
  PhiloxStep p;
  p.b = tag ^ K.k[0].y;
  p.c = (uint32_t)m1 ^ K.k[1].x;
  p.d = (uint32_t)(mA >> 32) ^ K.k[1].y;
  p.e = (uint32_t)mA ^ K.k[2].y;
  return p;
}

__device__ __forceinline__ Words4 philox_cell(uint32_t c, const PhiloxStep& p,
                                              const RoundKeys& K) {
  // round 0: word 0 is the cell, words 1-3 the step's
  const uint64_t m0 = (uint64_t)c * kPhiloxMul0;
  const uint32_t l0 = (uint32_t)m0;
  uint32_t x2 = (uint32_t)(m0 >> 32) ^ p.b;
  // round 1: word 0 is A, word 1 lo(step_hi M1)
  const uint64_t m1 = (uint64_t)x2 * kPhiloxMul1;
  uint32_t x0 = (uint32_t)(m1 >> 32) ^ p.c;
  uint32_t x1 = (uint32_t)m1;
  x2 = l0 ^ p.d;
  // round 2: word 3 is lo(A M0)
  uint32_t x3;
  {
    const uint64_t a = (uint64_t)x0 * kPhiloxMul0;
    const uint64_t b = (uint64_t)x2 * kPhiloxMul1;
    x0 = (uint32_t)(b >> 32) ^ x1 ^ K.k[2].x;
    x2 = (uint32_t)(a >> 32) ^ p.e;
    x1 = (uint32_t)b;
    x3 = (uint32_t)a;
  }
#pragma unroll
  for (int r = 3; r < 10; ++r) {
    const uint64_t a = (uint64_t)x0 * kPhiloxMul0;
    const uint64_t b = (uint64_t)x2 * kPhiloxMul1;
    const uint2 kr = K.k[r];
    const uint32_t y0 = (uint32_t)(b >> 32) ^ x1 ^ kr.x;
    const uint32_t y2 = (uint32_t)(a >> 32) ^ x3 ^ kr.y;
    x1 = (uint32_t)b;
    x3 = (uint32_t)a;
    x0 = y0;
    x2 = y2;
  }
  return Words4{x0, x1, x2, x3};
}

// The per-step parts of the sweep's draws (tag 0, and tag 1 with two words
// per update).
struct StepDraw {
  PhiloxStep acc, prop;
};

__host__ __device__ inline StepDraw step_draw(uint32_t step_lo, uint32_t step_hi,
                                              const RoundKeys& K) {
  return StepDraw{philox_step(step_lo, step_hi, kTagAccept, K),
                  philox_step(step_lo, step_hi, kTagPropose, K)};
}

// Cell word of the square lattice: sigma of arm a in bits [4a, 4a+3) (one
// nibble per arm, bits 4a+3 zero).
__device__ __forceinline__ uint32_t arm_of(uint32_t w, int a) {
  return (w >> (4 * a)) & 7u;
}

// The acceptance draws and proposal offsets of a cell from its Philox words.
// One word per update: w (q-1) = k 2^32 + u splits into the proposal offset k
// (high word) and the acceptance draw u (low word).  Two words per update:
// u from tag 0 (words u), k = floor(p (q-1) / 2^32) from tag 1 (words p).
template <int RNG_WORDS>
__device__ __forceinline__ void split_draws(const Words4& u, const Words4& p, uint32_t q,
                                            uint32_t acc[4], uint32_t kk[4]) {
  const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
  if (RNG_WORDS == 1) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const uint64_t prod = (uint64_t)uw[a] * (uint64_t)(q - 1u);
      kk[a] = (uint32_t)(prod >> 32);
      acc[a] = (uint32_t)prod;
    }
  } else {
    const uint32_t pw[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      acc[a] = uw[a];
      kk[a] = __umulhi(pw[a], q - 1u);
    }
  }
}

template <int RNG_WORDS>
__device__ __forceinline__ void cell_draws(uint32_t c, uint32_t step_lo,
                                           uint32_t step_hi, const RoundKeys& K,
                                           uint32_t q, uint32_t acc[4],
                                           uint32_t kk[4]) {
  const Words4 u = philox(c, step_lo, step_hi, kTagAccept, K);
  const Words4 p = (RNG_WORDS == 2) ? philox(c, step_lo, step_hi, kTagPropose, K) : u;
  split_draws<RNG_WORDS>(u, p, q, acc, kk);
}

// cell_draws with the step's parts of the draws folded in (step_draw).
template <int RNG_WORDS>
__device__ __forceinline__ void cell_draws_step(uint32_t c, const StepDraw& sd,
                                                const RoundKeys& K, uint32_t q, uint32_t acc[4],
                                                uint32_t kk[4]) {
  const Words4 u = philox_cell(c, sd.acc, K);
  const Words4 p = (RNG_WORDS == 2) ? philox_cell(c, sd.prop, K) : u;
  split_draws<RNG_WORDS>(u, p, q, acc, kk);
}

// Equal pairs among the four arms of a cell (its share of N_sigma).
__device__ __forceinline__ uint32_t cell_pairs(uint32_t w) {
  const uint32_t a0 = arm_of(w, 0), a1 = arm_of(w, 1), a2 = arm_of(w, 2),
                 a3 = arm_of(w, 3);
  return (uint32_t)(a0 == a1) + (uint32_t)(a0 == a2) + (uint32_t)(a0 == a3) +
         (uint32_t)(a1 == a2) + (uint32_t)(a1 == a3) + (uint32_t)(a2 == a3);
}

// ---------------------------------------------------------------------------
// FP64 part: Lennard-Jones energy per cell, volume move, observables.
// These must evaluate the same IEEE operations in the same order as any other
// implementation of the same readings; the library is compiled with
// -fmad=false so no multiply-add is contracted.
// ---------------------------------------------------------------------------
constexpr int kMaxShells = 256;

struct VolumeArgs {
  int64_t N;
  double epsilon, cutoff2;       // cutoff2: cutoff^2 (2D) or cutoff^6 (3D)
  double J, J_sigma, v_HB, kT, P;
  double dV_max;
  int32_t volume_moves;
  int32_t nshell;
  int32_t dim;                   // 3: cubic lattice; anything else: square lattice
  int32_t pad_dim;
  double shell_d2[kMaxShells];   // 2D: |d|^2 of the shells, ascending; 3D: |d|^6
  double S12[kMaxShells + 1];    // prefix sums of m / |d|^12 over the shells
  double S6[kMaxShells + 1];     // prefix sums of m / |d|^6
};

// 2D: u(v) = 2 eps [x^6 S12(n) - x^3 S6(n)], x = 1/v, n = number of shells
// with |d|^2 v < cutoff^2: the LJ energy per cell of a monolayer of lattice
// spacing sqrt(v) (half of each pair per cell), shell by shell.
// 3D: u(v) = 2 eps [x^4 S12(n) - x^2 S6(n)], n = number of shells with
// |d|^6 v^2 < cutoff^6: the cubic lattice of spacing r = v^(1/3) (Sec. II.A),
// tested without cube roots.
// The number n of shells inside the cutoff is found by bisection: the test
// (|d|^2 v < cutoff^2, or |d|^6 v v < cutoff^6) holds for a prefix of the
// ascending shells (IEEE products by a positive v keep their order), so n is
// the first shell where it fails -- the count a scan from the first shell
// gives, in about log2(nshell) dependent loads instead of n.
__device__ __forceinline__ int lj_shells_inside(const VolumeArgs& V, double v) {
  int lo = 0, hi = V.nshell;  // the test holds below lo and fails at hi
  const bool cubic = V.dim == 3;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const double key = cubic ? (V.shell_d2[mid] * v) * v : V.shell_d2[mid] * v;
    if (key < V.cutoff2)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// The same count with every lane of a warp testing its own shell: the test
// holds for a prefix of the shells, so the number of lanes where it holds,
// 32 shells at a time, is the bisection's result.  FP64 instructions occupy
// the pipe for a whole warp whatever the number of active lanes, so 32 tests
// cost what one does.  All 32 lanes call it.
__device__ __forceinline__ int lj_shells_inside_warp(const VolumeArgs& V, double v) {
  const int lane = (int)(threadIdx.x & 31u);
  const bool cubic = V.dim == 3;
  int n = 0;
  for (int base = 0; base < V.nshell; base += 32) {
    const int i = base + lane;
    bool in = false;
    if (i < V.nshell) {
      const double key = cubic ? (V.shell_d2[i] * v) * v : V.shell_d2[i] * v;
      in = key < V.cutoff2;
    }
    const unsigned int m = __ballot_sync(0xFFFFFFFFu, in);
    n += __popc(m);
    if (m != 0xFFFFFFFFu) break;
  }
  return n;
}

// u(v) from the number k of shells inside the cutoff.
__device__ __forceinline__ double lj_energy_at(const VolumeArgs& V, double v, int k) {
  if (V.dim == 3) {
    const double x = 1.0 / v;
    const double x2 = x * x;
    const double x4 = x2 * x2;
    return (2.0 * V.epsilon) * (x4 * V.S12[k] - x2 * V.S6[k]);
  }
  const double x = 1.0 / v;
  const double x3 = x * x * x;
  const double x6 = x3 * x3;
  return (2.0 * V.epsilon) * (x6 * V.S12[k] - x3 * V.S6[k]);
}

__device__ __forceinline__ double lj_cell_energy(const VolumeArgs& V, double v) {
  return lj_energy_at(V, v, lj_shells_inside(V, v));
}

// Block-wide copy of the FP64 parameters and shell tables into shared
// memory (the single thread that decides a volume move then reads them at
// shared-memory latency); the caller synchronises before using dst.
__device__ __forceinline__ void stage_volume_args(VolumeArgs* dst, const VolumeArgs* src) {
  static_assert(sizeof(VolumeArgs) % 8 == 0, "VolumeArgs copies as 64-bit words");
  const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(VolumeArgs) / 8); i += blockDim.x) d[i] = s[i];
}

__device__ __forceinline__ double u53(uint32_t hi, uint32_t lo) {
  const uint64_t m = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
  return (double)m * (1.0 / 9007199254740992.0);
}

// Device copy of the handle's scalar state.
struct Ctrl {
  // committed state after the last completed step
  long long sweep;
  long long n_hb_raw;
  long long n_coop;
  long long acc_sigma;
  long long acc_volume;
  double V_iso;
  double u_cell;        // u(V_iso / N)
  int g;
  int record_every;
  // the volume move of step `sweep` (already decided; its gate drives the
  // sigma sweep of that step)
  double next_V;
  double next_u;
  int next_g;
  int next_acc;
  // the volume move of step `sweep + 1`, decided early by the sweep kernel
  // when it does not depend on the bonds (ahead_state 1), or left to the end
  // of the step (ahead_state 0)
  double ahead_V;
  double ahead_u;
  int ahead_g;
  int ahead_acc;
  int ahead_state;
  int plan;             // cubic lattice: launch plan of the current step's six passes
  // per-step accumulators (zero between steps)
  unsigned long long acc_hb;
  unsigned long long acc_pairs;
  unsigned long long acc_moves;
  unsigned int done;
  unsigned int tile_next;
  // observable ring: records written so far (monotone)
  long long ring_head;
  // N_q' of the step being recorded (accumulated by the sweep only when its
  // observables go to the ring) and of the last recorded step
  unsigned long long acc_hist[8];
  long long hist[8];
  unsigned int error;  // nonzero: a bounded device-side wait gave up (bit 0), a
                       // debug-build index check failed (0x100 + site), or a
                       // lattice given to the sweep held an invalid cell
                       // (kStatusBadCell)
  unsigned int pad1;
};

// Status bit of a lattice that holds a word which is not a valid cell for q.
constexpr unsigned int kStatusBadCell = 0x200u;

struct VolumeResult {
  double V, u;
  int g, accepted;
};

// The volume move of MC step `step` (Sec. II.B step 1, with the oracle's
// readings): dV = (2 u1 - 1) dV_max from Philox((2^32-1, step, 3)); the hard
// core rejects v' < 1; the gate is g' = [v' < 2]; the enthalpy change is
// N (u(v') - u(v)) + P dV - (g' - g) J_eff N_HB_raw and the move is accepted
// when u2 < exp(-dH/kT + N ln(V'/V)).  When n_hb_raw < 0 (bonds not yet
// known) and the proposal would change the gate, returns false and decides
// nothing; otherwise fills *out and returns true.
__device__ __forceinline__ bool volume_decide(const VolumeArgs& V, long long step, double V_old,
                                              double u_old, int g, long long n_hb_raw,
                                              const RoundKeys& K, VolumeResult* out) {
  out->V = V_old;
  out->u = u_old;
  out->g = g;
  out->accepted = 0;
  if (!V.volume_moves) return true;
  const Words4 r = philox(kCellVolume, (uint32_t)((unsigned long long)step & 0xFFFFFFFFu),
                          (uint32_t)((unsigned long long)step >> 32), kTagVolume, K);
  const double u1 = u53(r.x, r.y);
  const double u2 = u53(r.z, r.w);
  const double Nd = (double)V.N;
  const double dV = (2.0 * u1 - 1.0) * V.dV_max;
  const double V_new = V_old + dV;
  const double v_new = V_new / Nd;
  if (v_new < 1.0) return true;
  const int g_new = (v_new < 2.0) ? 1 : 0;
  if (g_new != g && n_hb_raw < 0) return false;
  const double J_eff = V.J - V.P * V.v_HB;
  const double u_new = lj_cell_energy(V, v_new);
  const double du = u_new - u_old;
  const double t1 = Nd * du;
  const double t2 = V.P * dV;
  // with unknown bonds the gate is unchanged here, so the bond term is zero
  const double t3 = ((double)(g_new - g) * J_eff) * (double)(n_hb_raw < 0 ? 0 : n_hb_raw);
  const double dH = (t1 + t2) - t3;
  const double arg = -dH / V.kT + Nd * log(V_new / V_old);
  if (u2 < exp(arg)) {
    out->V = V_new;
    out->u = u_new;
    out->g = g_new;
    out->accepted = 1;
  }
  return true;
}

// volume_decide on two warps of one block, for the kernels that have two
// warps free while the lattice is swept.  FP64 instructions occupy the FP64
// pipe of a warp's SM sub-partition for a whole warp (64 cycles on GB300)
// whatever the number of active lanes, and warps w and w + 1 sit on
// different sub-partitions, so (a) the two divisions of the proposal, v' =
// V'/N and V'/V, run in lanes 0 and 1 of one pass, (b) the shells inside the
// cutoff are counted 32 at a time (lj_shells_inside_warp), and (c) warp
// role 1 takes log(V'/V) (the longest function here) while warp role 0
// evaluates the energy change; role 0 waits for it on named barrier BAR
// (64 threads) before the final exp.  The IEEE operations and their order
// are those of volume_decide, so the decision is identical.  Called by all
// 64 threads (role = 0 or 1 per warp) with the same arguments; xch is a
// shared double; the result in *out is valid in role 0's lanes.  The early
// returns depend only on values both warps compute alike, so either both
// reach the barrier or neither does.
template <int BAR>
__device__ __forceinline__ bool volume_decide_pair(int role, const VolumeArgs& V, long long step,
                                                   double V_old, double u_old, int g,
                                                   long long n_hb_raw, const RoundKeys& K,
                                                   VolumeResult* out, double* xch) {
  out->V = V_old;
  out->u = u_old;
  out->g = g;
  out->accepted = 0;
  if (!V.volume_moves) return true;
  const Words4 r = philox(kCellVolume, (uint32_t)((unsigned long long)step & 0xFFFFFFFFu),
                          (uint32_t)((unsigned long long)step >> 32), kTagVolume, K);
  const double u1 = u53(r.x, r.y);
  const double u2 = u53(r.z, r.w);
  const double Nd = (double)V.N;
  const double dV = (2.0 * u1 - 1.0) * V.dV_max;
  const double V_new = V_old + dV;
  const unsigned int lane = threadIdx.x & 31u;
  const double quot = V_new / ((lane == 1u) ? V_old : Nd);  // lane 0: v', lane 1: V'/V
  const double v_new = __shfl_sync(0xFFFFFFFFu, quot, 0);
  const double ratio = __shfl_sync(0xFFFFFFFFu, quot, 1);
  if (v_new < 1.0) return true;
  const int g_new = (v_new < 2.0) ? 1 : 0;
  if (g_new != g && n_hb_raw < 0) return false;
  if (role == 1) {
    const double lr = Nd * log(ratio);
    if (lane == 0u) *xch = lr;
    asm volatile("bar.sync %0, 64;" ::"n"(BAR) : "memory");
    return true;
  }
  const double J_eff = V.J - V.P * V.v_HB;
  const double u_new = lj_energy_at(V, v_new, lj_shells_inside_warp(V, v_new));
  const double du = u_new - u_old;
  const double t1 = Nd * du;
  const double t2 = V.P * dV;
  const double t3 = ((double)(g_new - g) * J_eff) * (double)(n_hb_raw < 0 ? 0 : n_hb_raw);
  const double dH = (t1 + t2) - t3;
  const double q = -dH / V.kT;
  asm volatile("bar.sync %0, 64;" ::"n"(BAR) : "memory");
  const double arg = q + *xch;
  if (u2 < exp(arg)) {
    out->V = V_new;
    out->u = u_new;
    out->g = g_new;
    out->accepted = 1;
  }
  return true;
}

// Observables of the committed state (Eq. V and Eq. H).
__device__ __forceinline__ cvf_obs make_obs(const VolumeArgs& V, const Ctrl* ctl) {
  cvf_obs o;
  const double Nd = (double)V.N;
  const long long nhb = ctl->g ? ctl->n_hb_raw : 0;
  const double U = Nd * ctl->u_cell;
  const double vol = ctl->V_iso + V.v_HB * (double)nhb;
  const double H = ((U - V.J * (double)nhb) - V.J_sigma * (double)ctl->n_coop) + V.P * vol;
  o.sweep = ctl->sweep;
  o.n_hb = nhb;
  o.n_hb_raw = ctl->n_hb_raw;
  o.n_coop = ctl->n_coop;
  o.acc_sigma = ctl->acc_sigma;
  o.acc_volume = ctl->acc_volume;
  o.V_iso = ctl->V_iso;
  o.V = vol;
  o.U_LJ = U;
  o.H = H;
  o.g = ctl->g;
  o.status = (int32_t)ctl->error;
  for (int v = 0; v < 8; ++v) o.n_state[v] = ctl->hist[v];
  return o;
}

// End of a step, run by one thread once every block's counts are in:
// commit the counts and the step's volume move, advance the step counter,
// append the observables to the ring when the step count is a multiple of
// record_every, and settle the volume move of the next step (taken from the
// early decision when there is one, else decided now with the new bonds).
// All accesses go through a volatile view: in the batched kernel the
// previous step of the same lattice was closed by another SM without a
// kernel boundary in between.
// DELTA = false: acc_hb / acc_pairs hold the step's totals (the square
// lattice recounts its bonds in every sweep).  DELTA = true: they hold the
// changes made by the accepted moves (two's complement), added to the
// committed counts (the cubic lattice's layered passes).
template <bool DELTA = false>
__device__ __forceinline__ void finalize_step(const VolumeArgs& V, Ctrl* ctl, cvf_obs* ring,
                                              long long ring_cap, const RoundKeys& K) {
  volatile Ctrl* c = ctl;
  // Every field the commit reads is loaded before the first store, so the
  // loads are in flight together (one memory round trip on the step's
  // critical path); the early decision's fields are used only when
  // ahead_state says they hold one.
  const int every = c->record_every;
  const long long sweep = c->sweep;
  const long long n_hb_raw = c->n_hb_raw, n_coop = c->n_coop;
  const long long acc_sigma = c->acc_sigma, acc_volume = c->acc_volume;
  const unsigned long long acc_hb = c->acc_hb, acc_pairs = c->acc_pairs,
                           acc_moves = c->acc_moves;
  const double next_V = c->next_V, next_u = c->next_u;
  const int next_g = c->next_g, next_acc = c->next_acc;
  const int ahead = c->ahead_state;
  const double ahead_V = c->ahead_V, ahead_u = c->ahead_u;
  const int ahead_g = c->ahead_g, ahead_acc = c->ahead_acc;
  const long long head = c->ring_head;
  Ctrl s;  // committed state after this step
  const bool recorded = (every > 0) && ((sweep + 1) % every == 0);
  if (DELTA) {
    s.n_hb_raw = n_hb_raw + (long long)acc_hb;
    s.n_coop = n_coop + (long long)acc_pairs;
  } else {
    s.n_hb_raw = (long long)acc_hb;
    // N_sigma is counted by the sweep only on recorded steps; otherwise it is
    // unknown (-1) until a recount (cvf_observables counts it on demand)
    s.n_coop = recorded ? (long long)acc_pairs : -1;
  }
  s.acc_sigma = acc_sigma + (long long)acc_moves;
  s.V_iso = next_V;
  s.u_cell = next_u;
  s.g = next_g;
  s.acc_volume = acc_volume + next_acc;
  s.sweep = sweep + 1;
  c->n_hb_raw = s.n_hb_raw;
  c->n_coop = s.n_coop;
  c->acc_sigma = s.acc_sigma;
  c->V_iso = s.V_iso;
  c->u_cell = s.u_cell;
  c->g = s.g;
  c->acc_volume = s.acc_volume;
  c->acc_hb = 0;
  c->acc_pairs = 0;
  c->acc_moves = 0;
  c->done = 0;
  c->tile_next = 0;
  c->sweep = s.sweep;
  if (recorded) {
    s.error = c->error;  // the record's status word
    for (int v = 0; v < 8; ++v) {
      s.hist[v] = (long long)c->acc_hist[v];
      c->hist[v] = s.hist[v];
      c->acc_hist[v] = 0;
    }
    ring[head % ring_cap] = make_obs(V, &s);
    c->ring_head = head + 1;
  }
  VolumeResult r;
  if (ahead == 1) {
    r.V = ahead_V;
    r.u = ahead_u;
    r.g = ahead_g;
    r.accepted = ahead_acc;
  } else {
    volume_decide(V, s.sweep, s.V_iso, s.u_cell, s.g, s.n_hb_raw, K, &r);
  }
  c->next_V = r.V;
  c->next_u = r.u;
  c->next_g = r.g;
  c->next_acc = r.accepted;
  c->ahead_state = 0;
}

// Programmatic dependent launch (sm_90 and later): a kernel launched with
// programmatic stream serialization may start while the previous kernel of
// the stream still runs -- once every block of that kernel has called
// pdl_trigger or exited -- and pdl_wait blocks until the previous kernel has
// completed and its writes are visible.  A kernel that calls pdl_wait before
// any global access computes exactly what it computes after a plain launch;
// only the launch latency overlaps the previous kernel's tail.  Both are
// no-ops for a plain launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Atomic add with acquire-release semantics at GPU scope: the caller's
// earlier writes (and, after a block barrier, its block's) are visible to
// whoever acquires a later value of the counter, and the caller sees every
// write released before the values it adds to.
__device__ __forceinline__ unsigned int atom_add_acq_rel(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v)
               : "memory");
  return old;
}

// True in every thread of the block that arrives last (after all blocks
// have published their atomics).
__device__ __forceinline__ bool last_block(unsigned int* done) {
  __shared__ int is_last;
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atom_add_acq_rel(done, 1u) == gridDim.x - 1) ? 1 : 0;
  __syncthreads();
  return is_last != 0;
}

// True when the observables after step `step` (0-based, so the count after
// it is step + 1) go to the ring: the sweep then also accumulates N_q'.
__device__ __forceinline__ bool step_recorded(int every, long long step) {
  return every > 0 && (step + 1) % every == 0;
}

// N_q' of the cells a block finishes, accumulated only on recorded steps in
// four shared words: lane v & 3 (16 bits) of word v & 3, v < 4 in the low
// half, v >= 4 in the high half, from each cell's count word (nibble v =
// number of the cell's arms with sigma = v).  A tile adds at most 4 x 8192
// to a lane; the words are moved to the 64-bit totals after every tile.
__device__ __forceinline__ void hist_add_cell(uint32_t* s_hist4, uint32_t cnt) {
  atomicAdd(&s_hist4[0], cnt & 0x000F000Fu);
  atomicAdd(&s_hist4[1], (cnt >> 4) & 0x000F000Fu);
  atomicAdd(&s_hist4[2], (cnt >> 8) & 0x000F000Fu);
  atomicAdd(&s_hist4[3], (cnt >> 12) & 0x000F000Fu);
}

// Called by the whole block after its shared adds are complete (after a
// barrier): moves the four words to out[0..8) and clears them.
__device__ __forceinline__ void hist_flush(uint32_t* s_hist4, unsigned long long* out) {
  if (threadIdx.x < 4) {
    const uint32_t w = s_hist4[threadIdx.x];
    if (w & 0xFFFFu) atomicAdd(&out[threadIdx.x], (unsigned long long)(w & 0xFFFFu));
    if (w >> 16) atomicAdd(&out[threadIdx.x + 4], (unsigned long long)(w >> 16));
    s_hist4[threadIdx.x] = 0;
    __threadfence();  // visible before the block reports itself done
  }
}

// Block-wide sum of three counters; the result is valid in thread 0.
template <int NT>
__device__ __forceinline__ void block_sum3(uint32_t& a, uint32_t& b, uint32_t& c) {
  __shared__ uint32_t red[3][NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xFFFFFFFFu, a, o);
    b += __shfl_xor_sync(0xFFFFFFFFu, b, o);
    c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = a;
    red[1][wid] = b;
    red[2][wid] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = 0; b = 0; c = 0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) {
      a += red[0][i];
      b += red[1][i];
      c += red[2][i];
    }
  }
}

// ---------------------------------------------------------------------------
// Debug builds (compiled with CVF_DEBUG): device-side index checks in place
// of a memory checker.  dcheck(ok, err, site) records the first failing
// check of a launch in the lattice's error word as 0x100 + site and returns
// false, and the caller skips the access instead of faulting; in release
// builds it is the constant true and the checks compile away.
// ---------------------------------------------------------------------------
enum DebugSite : unsigned int {
  kSiteStage = 1,       // staged tile: source row / word and shared-memory slot
  kSiteTma = 2,         // TMA box: 16-byte aligned x and the box inside the lattice
  kSiteTileRead = 3,    // colour phases: shared-memory reads of the staged tile
  kSiteTileWrite = 4,   // colour phases: shared-memory and global writes
  kSitePass3 = 5,       // cubic passes: the cell group and its neighbour words
  kSiteResident2 = 6,   // square lattice resident in one cluster
  kSiteResident3 = 7,   // cubic lattice resident in one cluster
  kSiteBatchItem = 8,   // batched sweep: decoded replica and tile of a work item
  kSiteLayer = 9,       // layered square-lattice passes
  kSiteEta3 = 10,       // cubic lattice: cube moves and eta copies
};

#ifdef CVF_DEBUG
__device__ __forceinline__ bool dcheck(bool ok, unsigned int* err, unsigned int site) {
  if (!ok && err) atomicCAS(err, 0u, 0x100u + site);
  return ok;
}
#else
__device__ __forceinline__ constexpr bool dcheck(bool, unsigned int*, unsigned int) {
  return true;
}
#endif

// ---------------------------------------------------------------------------
// Bounded waits.  A thread that waits for another block (the persistent
// batched sweep: a tile of step s waits until its replica finished step
// s - 1) polls with acquire loads and a short sleep, and gives up after a
// fixed number of polls, so that a wait that can never end returns an error
// status instead of hanging the GPU.
// ---------------------------------------------------------------------------
constexpr unsigned int kWaitPollLimit = 1u << 22;  // about half a second of sleep

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

enum WaitResult { kWaitDone = 0, kWaitGaveUp = 1, kWaitAborted = 2 };

// Poll until *flag >= target; stop early when *abort_word becomes nonzero
// (another block gave up).  A waiter d steps short of its target sleeps about
// 128 min(d, 8)^2 ns between polls, so blocks that took work far ahead (a
// small lattice's later steps) leave the memory system to the ones about to
// run; one step short it polls every 128 ns.  Each poll is charged its sleep
// in 128-ns quanta, and the wait gives up once `limit` quanta are used (one
// per poll when d = 1).
__device__ __forceinline__ WaitResult wait_flag_geq(const unsigned int* flag, unsigned int target,
                                                    const unsigned int* abort_word,
                                                    unsigned int limit) {
  unsigned int used = 0;
  for (;;) {
    const unsigned int v = ld_acquire(flag);
    if (v >= target) return kWaitDone;
    if (abort_word && *(volatile const unsigned int*)abort_word) return kWaitAborted;
    const unsigned int d = min(target - v, 8u);
    used += d * d;
    if (used > limit) return kWaitGaveUp;
    __nanosleep(128u * d * d);
  }
}

}  // namespace cvf
