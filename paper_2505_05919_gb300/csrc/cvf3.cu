// cvf3.cu -- the paper's own 3D CVF Metropolis (arXiv:2505.05919, Sec. II):
// a periodic cubic lattice, six bonding indices per cell, one nibble each in
// one uint32 word, the layered partition of Sec. II.C (the six arm
// domains updated one after the other in an order drawn every MC step), the
// counts of Eq. (H) kept incrementally, and the isobaric volume move of
// Sec. II.B with the cubic-lattice Lennard-Jones energy.
//
// eta (App. A).  The checkerboard cubes are the unit cells whose corner of
// smallest coordinates has all three coordinates even or all odd; they
// partition the edges, and each cube's eta = 0 edges are one of the nine
// perfect matchings of the cube graph (its configuration, one byte per cube
// in `eta`).  The configurations are the state; every cell word also keeps
// a copy of the eta of its six edges in the spare bit 3 of each arm's
// nibble (1 = allowed), so that a pass reads it with the cell.  Step 2 of
// the MC step (k_eta3, one thread per cube) moves every cube and flips the
// copies at its corners by atomic XOR; the arm rule then drops the bond term
// of an edge with eta = 0.  Without eta moves every copy is 1.
//
// Launch structure.  A pass over arm a reads, besides the cell's own word,
// only arm a^1 of the neighbour in direction a.  That arm changes only in
// the pass over a^1.  So consecutive passes whose arms contain no opposite
// pair can run in one launch, each thread taking its cells through all of
// them in registers: every neighbour arm it reads is constant during the
// launch, whichever version of the neighbour's word it sees, and the result
// is the one of the passes run one after the other.  The six passes of a
// step are cut greedily before the first arm whose opposite is already in
// the current launch, which gives 2 to 4 launches (2.67 on average over the
// 720 orders); every step enqueues four launches, the unused ones return at
// once, and the fourth commits the step.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "cvf_device.cuh"
#include "cvf_fastdiv.cuh"
#include "cvf_host.h"
#include "cvf_lattice.cuh"

namespace cg = cooperative_groups;

namespace cvf {
namespace {

constexpr int kThreads3 = 256;
constexpr int kLaunches3 = 4;           // launches per MC step (most segments)
constexpr int kGraphSteps3 = 32;
constexpr long long kRingCap3 = 65536;
constexpr uint32_t kTagArm0 = 8u;       // draws of arm a: Philox tag 8 + a
constexpr uint32_t kTagInit0 = 16u;     // random init of arm a: tag 16 + a
constexpr uint32_t kR7 = 0x1111111u;    // 1 in nibbles 0..6
constexpr uint32_t kM7 = 0x8888888u;    // bit 3 of nibbles 0..6
constexpr uint32_t kArmBits = 0x777777u;  // the sigma bits of the six arm nibbles
constexpr uint32_t kEtaBits = 0x888888u;  // bit 3 of the six arm nibbles: the edges' eta
constexpr uint32_t kTagEta = 5u;          // cube moves: Philox tag 5
constexpr uint32_t kTagEtaInit = 6u;      // random initial cube configurations: tag 6
constexpr int kMaxSide3 = 1024;

struct Args3 {
  uint32_t* state;                  // L^3 words, updated in place
  Ctrl* ctrl;
  const unsigned long long* table;  // [g][(dN_HB+1)*11 + dN_sigma+5]
  const VolumeArgs* vol;
  cvf_obs* ring;
  long long ring_cap;
  RoundKeys keys;
  uint32_t L, L2, N;
  uint32_t groups;                  // ceil(N / 4): four consecutive cells each
  uint32_t G;                       // L / 4 (groups per row when L % 4 == 0)
  uint32_t q;
  FastDiv div_G, div_L, div_L2;
  // eta (App. A): cube configurations (L^3/4 bytes; null without eta moves),
  // the 12-bit edge masks of the nine configurations, the move thresholds
  // [g][dN_HB + 4], L / 2 and the number of cubes
  uint8_t* eta;
  const unsigned long long* eta_table;
  uint16_t masks[9];
  uint32_t H, ncube;
  FastDiv div_H;
};

// ---------------------------------------------------------------------------
// Arm order and launch plan of a step.  The order is permutation number
// floor(w 720 / 2^32) of the six arms (lexicographic), w word 0 of
// Philox((2^32-2, step, 4)).  Plan word: bits 3i..3i+2 the arm of pass i,
// bit 17 + i set when pass i opens a new launch (i = 1..5).
// ---------------------------------------------------------------------------
__device__ uint32_t make_plan(long long step, const RoundKeys& K) {
  const Words4 r = philox(kCellLayers, (uint32_t)((unsigned long long)step & 0xFFFFFFFFu),
                          (uint32_t)((unsigned long long)step >> 32), kTagLayers, K);
  uint32_t idx = __umulhi(r.x, 720u);
  int avail[6] = {0, 1, 2, 3, 4, 5};
  const uint32_t fact[6] = {120u, 24u, 6u, 2u, 1u, 1u};
  uint32_t plan = 0, in_launch = 0;
  int left = 6;
  for (int i = 0; i < 6; ++i) {
    const uint32_t j = idx / fact[i];
    idx -= j * fact[i];
    const int a = avail[j];
    for (int t = (int)j; t < left - 1; ++t) avail[t] = avail[t + 1];
    --left;
    if (in_launch & (1u << (a ^ 1))) {
      plan |= 1u << (17 + i);
      in_launch = 0;
    }
    in_launch |= 1u << a;
    plan |= (uint32_t)a << (3 * i);
  }
  return plan;
}

__device__ __forceinline__ int plan_launches(uint32_t plan) { return 1 + __popc(plan >> 18); }

// Arms of launch j of the plan (at most three: no opposite pair).
__device__ int plan_arms(uint32_t plan, int j, int* arms) {
  int launch = 0, n = 0;
  for (int i = 0; i < 6; ++i) {
    if (i > 0 && ((plan >> (17 + i)) & 1u)) ++launch;
    if (launch == j && n < 3) arms[n++] = (int)((plan >> (3 * i)) & 7u);
  }
  return n;
}

// ---------------------------------------------------------------------------
// Metropolis update of arm a of one cell (Sec. II.C with Eq. H).
//   w     the cell word (sigma_b in nibble b), nw the neighbour's word in
//         direction a (its nibble a^1 is the partner arm), r the cell's draw
//   sh    4a; nsh = 24 - 4 (a^1) moves the partner nibble to nibble 6;
//   amask 0xF << 4a
// Proposal: w (q-1) = k 2^32 + u, sigma' from the shared table
// prop[8 sigma + k] = ((sigma + 1 + k) mod q) * 0x1111111 (sigma' in nibbles
// 0..6).  With the partner in nibble 6 of wn, f(v) = (((wn ^ v R) | M) - R)
// & M has bit 3 of nibble b set iff nibble b differs from v (no borrow
// crosses a nibble since every nibble is >= 8 before the subtraction).  So
// popc f(sigma) = A_s + b_s and popc f(sigma') = A_p + b_p, with A_v the arms
// differing from v and b_v = [partner != v] (bit 27); dN_HB = b_s - b_p and
// dN_sigma = A_s - A_p + 1, and the threshold row index
// 11 dN_HB + dN_sigma + 16 = (popc f_s + 10 b_s) - (popc f_p + 10 b_p) + 17.
// The row holds {T - 1, packed count change}; an accepted move adds the
// latter ((1 << 24) + ((dN_HB + 1) << 16) + dN_sigma + 5) to pk.
// ---------------------------------------------------------------------------
struct Row3 {
  uint32_t t;      // T - 1 (every T >= 1 on this path) or unused (64-bit path)
  uint32_t delta;  // packed count change of an accepted move
};

// eta: bit 4a+3 of w (the copy of the edge's eta) moved to bit 27; when it
// is 0 the mask drops the partner's flag from both nibble tests, so b_s =
// b_p = 0, dN_HB = 0 and the row is the one of the arms alone.
template <bool CMP64>
__device__ __forceinline__ uint32_t update_arm3(uint32_t w, uint32_t nw, uint32_t r, uint32_t sh,
                                                uint32_t nsh, uint32_t amask, uint32_t qm1,
                                                const uint32_t* prop, const Row3* rows,
                                                const unsigned long long* T64, uint32_t& pk) {
  const uint32_t s = (w >> sh) & 7u;
  const uint32_t k = __umulhi(r, qm1);
  const uint32_t u = r * qm1;
  const uint32_t sR = s * kR7;
  const uint32_t spR = prop[s * 8u + k];
  const uint32_t wn = w | ((nw << nsh) & 0x7000000u);
  const uint32_t meta = ((w << (24u - sh)) & 0x8000000u) | 0x0888888u;
  const uint32_t fs = (((wn ^ sR) | kM7) - kR7) & meta;
  const uint32_t fp = (((wn ^ spR) | kM7) - kR7) & meta;
  const int idx = (int)(__popc(fs) + 10u * (fs >> 27)) - (int)(__popc(fp) + 10u * (fp >> 27)) + 17;
  const Row3 row = rows[idx];
  const bool accept = CMP64 ? ((unsigned long long)u < T64[idx]) : (u <= row.t);
  if (accept) {
    w ^= (sR ^ spR) & amask;
    pk += row.delta;
  }
  return w;
}

// Adds a group's packed count changes to the thread's totals.
__device__ __forceinline__ void unpack_counts(uint32_t& pk, uint32_t& nacc, uint32_t& hb_b,
                                              uint32_t& dc_b) {
  nacc += pk >> 24;
  hb_b += (pk >> 16) & 0xFFu;
  dc_b += pk & 0xFFFFu;
  pk = 0;
}

// N_q' of the four final cell words of a group, added to the block's eight
// shared counters: per word a count word (nibble v = arms in state v), two
// words summed (nibbles <= 12), nibbles v and v+4 moved to the 16-bit lanes
// of word v (<= 24 per lane), reduced over the converged lanes of the warp
// (<= 768 per lane) and added by the lowest of them.
__device__ __forceinline__ uint32_t count_word(uint32_t w) {
  uint32_t c = 0;
#pragma unroll
  for (int b = 0; b < 6; ++b) c += 1u << (4u * ((w >> (4 * b)) & 7u));
  return c;
}

__device__ __forceinline__ void hist_group(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3,
                                           uint32_t* s_hist) {
  const uint32_t h01 = count_word(w0) + count_word(w1);
  const uint32_t h23 = count_word(w2) + count_word(w3);
  const unsigned mask = __activemask();
  const int leader = __ffs(mask) - 1;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    uint32_t lanes = ((h01 >> (4 * v)) & 0x000F000Fu) + ((h23 >> (4 * v)) & 0x000F000Fu);
    lanes = __reduce_add_sync(mask, lanes);
    if ((int)(threadIdx.x & 31) == leader) {
      if (lanes & 0xFFFFu) atomicAdd(&s_hist[v], lanes & 0xFFFFu);
      if (lanes >> 16) atomicAdd(&s_hist[v + 4], lanes >> 16);
    }
  }
}

// ---------------------------------------------------------------------------
// One launch of a step.  ALIGNED: L % 4 == 0, a group (four consecutive
// cells) lies in one row, its words and its y/z neighbours' words are
// 16-byte vectors.  Otherwise every cell computes its own coordinates.
// Launch 0 has one extra block (block 0) that decides the next step's volume
// move early when it cannot depend on the bonds (no gate change); launch
// kLaunches3 - 1 commits the step.
// ---------------------------------------------------------------------------
template <bool ALIGNED, bool CMP64>
__global__ void __launch_bounds__(kThreads3, 4) k_pass3(Args3 A, int launch) {
  __shared__ Row3 sRows[33];
  __shared__ uint32_t sProp[64];
  __shared__ unsigned long long sT64[CMP64 ? 33 : 1];
  __shared__ int s_arm[3];
  __shared__ int s_n, s_rec;
  __shared__ uint32_t s_hist[8];
  Ctrl* ctl = A.ctrl;
  const bool fin = (launch == kLaunches3 - 1);
  if (threadIdx.x == 0) {
    uint32_t plan;
    if (launch == 0) {
      plan = make_plan(ctl->sweep, A.keys);
      if (blockIdx.x == 0) ctl->plan = (int)plan;
    } else {
      plan = (uint32_t)ctl->plan;
    }
    int arms[3] = {0, 0, 0};
    const int n = plan_arms(plan, launch, arms);
    s_n = n;
    for (int i = 0; i < 3; ++i) s_arm[i] = arms[i];
    // N_q' is accumulated by the launch that finishes a recorded step
    s_rec = (n > 0 && launch == plan_launches(plan) - 1 &&
             step_recorded(ctl->record_every, ctl->sweep)) ? 1 : 0;
  }
  __syncthreads();
  const int n_arms = s_n;
  if (launch == 0 && blockIdx.x == 0) {
    __shared__ VolumeArgs sV;  // the parameters at shared-memory latency
    __shared__ double s_xch;
    stage_volume_args(&sV, A.vol);
    __syncthreads();
    if (threadIdx.x < 64) {  // warps 0 and 1: the move on two FP64 pipes
      VolumeResult r;
      const bool ok = volume_decide_pair<3>((int)(threadIdx.x >> 5), sV, ctl->sweep + 1,
                                            ctl->next_V, ctl->next_u, ctl->next_g, -1, A.keys,
                                            &r, &s_xch);
      if (threadIdx.x == 0 && ok) {
        ctl->ahead_V = r.V;
        ctl->ahead_u = r.u;
        ctl->ahead_g = r.g;
        ctl->ahead_acc = r.accepted;
        ctl->ahead_state = 1;
      }
    }
    return;
  }
  if (n_arms == 0) {
    // nothing to update in this launch; the last one still commits the step
    if (fin && blockIdx.x == 0 && threadIdx.x == 0)
      finalize_step<true>(*A.vol, ctl, A.ring, A.ring_cap, A.keys);
    return;
  }
  const long long step = ctl->sweep;
  const int g = ctl->next_g;
  const bool rec = s_rec != 0;
  const uint32_t q = A.q;
  if (threadIdx.x < 33) {
    const unsigned long long t = A.table[g * 33 + threadIdx.x];
    if (CMP64) sT64[threadIdx.x] = t;
    const int dhb = (int)threadIdx.x / 11 - 1, dc = (int)threadIdx.x % 11 - 5;
    sRows[threadIdx.x].t = (uint32_t)(t - 1ull);  // every t >= 1 unless CMP64
    sRows[threadIdx.x].delta = (1u << 24) + ((uint32_t)(dhb + 1) << 16) + (uint32_t)(dc + 5);
  } else if (threadIdx.x >= 64 && threadIdx.x < 128) {
    const uint32_t s = (threadIdx.x - 64) >> 3, k = (threadIdx.x - 64) & 7u;
    uint32_t sp = s + 1u + k;
    while (sp >= q) sp -= q;
    sProp[threadIdx.x - 64] = (s < q && k + 1u < q) ? sp * kR7 : 0u;
  }
  if (threadIdx.x < 8) s_hist[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t s_lo = (uint32_t)((unsigned long long)step & 0xFFFFFFFFu);
  const uint32_t s_hi = (uint32_t)((unsigned long long)step >> 32);
  const uint32_t qm1 = q - 1u;
  const uint32_t first_block = (launch == 0) ? 1u : 0u;
  const uint32_t nblk = gridDim.x - first_block;
  // accepted moves and the biased sums of their dN_HB + 1 and dN_sigma + 5
  uint32_t nacc = 0, hb_b = 0, dc_b = 0, pk = 0;
  uint32_t* __restrict__ st = A.state;
  const uint32_t stride = nblk * kThreads3;
  const uint32_t g_first = (blockIdx.x - first_block) * kThreads3 + threadIdx.x;
  if (ALIGNED) {
    // The group loop is compiled once per number of passes in the launch and
    // once more for recorded steps (N_q' counted), so that the others carry
    // no per-group test of the flag (at 260^3: 479 against 449
    // sigma-updates/ns with the test inside the loop).
    // Pass p's neighbour word is at c0 + dlt - (coordinate == edge ? wrp : 0)
    // with the coordinate (x group, y or z), the edge value, the offset and
    // the periodic wrap fixed for the launch.
    auto body = [&](auto na_c, auto rec_c) {
      constexpr int NA = decltype(na_c)::value;
      constexpr bool REC = decltype(rec_c)::value;
      int arm[NA];
      uint32_t ax[NA], edge[NA], dlt[NA], wrp[NA];
#pragma unroll
      for (int p = 0; p < NA; ++p) {
        const int a = s_arm[p];
        arm[p] = a;
        const bool plus = (a & 1) == 0;
        if (a < 2) {
          ax[p] = 0u;
          edge[p] = plus ? A.G - 1u : 0u;
          dlt[p] = plus ? 4u : 0u - 1u;
          wrp[p] = plus ? A.L : 0u - A.L;
        } else if (a < 4) {
          ax[p] = 1u;
          edge[p] = plus ? A.L - 1u : 0u;
          dlt[p] = plus ? A.L : 0u - A.L;
          wrp[p] = plus ? A.L2 : 0u - A.L2;
        } else {
          ax[p] = 2u;
          edge[p] = plus ? A.L - 1u : 0u;
          dlt[p] = plus ? A.L2 : 0u - A.L2;
          wrp[p] = plus ? A.N : 0u - A.N;
        }
      }
      uint4 next = make_uint4(0u, 0u, 0u, 0u);
      if (g_first < A.groups) next = *reinterpret_cast<const uint4*>(st + 4u * g_first);
      for (uint32_t gi = g_first; gi < A.groups; gi += stride) {
        const uint32_t c0 = gi * 4u;
        if (!dcheck(c0 + 3u < A.N, &ctl->error, kSitePass3)) break;
        const uint4 own = next;
        if (gi + stride < A.groups) next = *reinterpret_cast<const uint4*>(st + 4u * (gi + stride));
        const uint32_t row = fdiv(gi, A.div_G);      // y + L z
        const uint32_t xg = gi - row * A.G;
        const uint32_t z = fdiv(row, A.div_L);
        const uint32_t y = row - z * A.L;
        uint4 nbv[NA];
#pragma unroll
        for (int p = 0; p < NA; ++p) {
          const uint32_t coord = (ax[p] == 0u) ? xg : ((ax[p] == 1u) ? y : z);
          const uint32_t off = c0 + dlt[p] - ((coord == edge[p]) ? wrp[p] : 0u);
          if (arm[p] >= 2) {
            nbv[p] = dcheck((off & 3u) == 0u && off + 3u < A.N, &ctl->error, kSitePass3)
                         ? *reinterpret_cast<const uint4*>(st + off)
                         : make_uint4(0u, 0u, 0u, 0u);
          } else {
            // arm a^1 of a neighbour is constant during the launch, so the
            // cell's own words as loaded serve for the x neighbours
            const uint32_t xw = dcheck(off < A.N, &ctl->error, kSitePass3) ? st[off] : 0u;
            nbv[p] = (arm[p] == 0) ? make_uint4(own.y, own.z, own.w, xw)
                                   : make_uint4(xw, own.x, own.y, own.z);
          }
        }
        uint32_t w0 = own.x, w1 = own.y, w2 = own.z, w3 = own.w;
#pragma unroll
        for (int p = 0; p < NA; ++p) {
          const int a = arm[p];
          const uint32_t sh = 4u * (uint32_t)a, nsh = 24u - 4u * (uint32_t)(a ^ 1);
          const uint32_t amask = 0xFu << sh;
          const Words4 r = philox(gi, s_lo, s_hi, kTagArm0 + (uint32_t)a, A.keys);
          w0 = update_arm3<CMP64>(w0, nbv[p].x, r.x, sh, nsh, amask, qm1, sProp, sRows, sT64, pk);
          w1 = update_arm3<CMP64>(w1, nbv[p].y, r.y, sh, nsh, amask, qm1, sProp, sRows, sT64, pk);
          w2 = update_arm3<CMP64>(w2, nbv[p].z, r.z, sh, nsh, amask, qm1, sProp, sRows, sT64, pk);
          w3 = update_arm3<CMP64>(w3, nbv[p].w, r.w, sh, nsh, amask, qm1, sProp, sRows, sT64, pk);
        }
        unpack_counts(pk, nacc, hb_b, dc_b);
        *reinterpret_cast<uint4*>(st + c0) = make_uint4(w0, w1, w2, w3);
        if (REC) hist_group(w0, w1, w2, w3, s_hist);
      }
    };
    auto arms = [&](auto rec_c) {
      if (n_arms == 1)
        body(std::integral_constant<int, 1>{}, rec_c);
      else if (n_arms == 2)
        body(std::integral_constant<int, 2>{}, rec_c);
      else
        body(std::integral_constant<int, 3>{}, rec_c);
    };
    if (rec)
      arms(std::true_type{});
    else
      arms(std::false_type{});
  } else {
    for (uint32_t gi = g_first; gi < A.groups; gi += stride) {
      const uint32_t c0 = gi * 4u;
      uint32_t w[4], x[4], y[4], z[4];
      bool valid[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const uint32_t c = c0 + (uint32_t)i;
        valid[i] = c < A.N;
        const uint32_t cc = valid[i] ? c : 0u;
        z[i] = fdiv(cc, A.div_L2);
        const uint32_t rem = cc - z[i] * A.L2;
        y[i] = fdiv(rem, A.div_L);
        x[i] = rem - y[i] * A.L;
        w[i] = valid[i] ? st[c] : 0u;
      }
      for (int p = 0; p < n_arms; ++p) {
        const int a = s_arm[p];
        const uint32_t sh = 4u * (uint32_t)a, nsh = 24u - 4u * (uint32_t)(a ^ 1);
        const uint32_t amask = 0xFu << sh;
        const Words4 r = philox(gi, s_lo, s_hi, kTagArm0 + (uint32_t)a, A.keys);
        const uint32_t rw[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (!valid[i]) continue;
          const uint32_t c = c0 + (uint32_t)i;
          uint32_t nb;
          if (a == 0)
            nb = (x[i] + 1u == A.L) ? c + 1u - A.L : c + 1u;
          else if (a == 1)
            nb = (x[i] == 0u) ? c + A.L - 1u : c - 1u;
          else if (a == 2)
            nb = (y[i] + 1u == A.L) ? c + A.L - A.L2 : c + A.L;
          else if (a == 3)
            nb = (y[i] == 0u) ? c + A.L2 - A.L : c - A.L;
          else if (a == 4)
            nb = (z[i] + 1u == A.L) ? c + A.L2 - A.N : c + A.L2;
          else
            nb = (z[i] == 0u) ? c + A.N - A.L2 : c - A.L2;
          if (!dcheck(nb < A.N, &ctl->error, kSitePass3)) continue;
          w[i] = update_arm3<CMP64>(w[i], st[nb], rw[i], sh, nsh, amask, qm1, sProp, sRows,
                                    sT64, pk);
        }
      }
      unpack_counts(pk, nacc, hb_b, dc_b);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (valid[i]) st[c0 + (uint32_t)i] = w[i];
      if (rec) {
        // cells past the end hold word 0, counted as six arms in state 0
        hist_group(w[0], w[1], w[2], w[3], s_hist);
        if (!valid[1] || !valid[2] || !valid[3]) {
          // a zero word counts six arms in state 0: take them back
          const uint32_t missing = (uint32_t)(!valid[1]) + (uint32_t)(!valid[2]) + (uint32_t)(!valid[3]);
          atomicSub(&s_hist[0], 6u * missing);
        }
      }
    }
  }
  uint32_t a1 = hb_b - nacc, a2 = dc_b - 5u * nacc, a3 = nacc;  // two's complement sums
  block_sum3<kThreads3>(a1, a2, a3);
  if (threadIdx.x == 0) {
    atomicAdd(&ctl->acc_hb, (unsigned long long)(long long)(int)a1);
    atomicAdd(&ctl->acc_pairs, (unsigned long long)(long long)(int)a2);
    atomicAdd(&ctl->acc_moves, (unsigned long long)a3);
  }
  if (rec) {
    __syncthreads();
    if (threadIdx.x < 8 && s_hist[threadIdx.x])
      atomicAdd(&ctl->acc_hist[threadIdx.x], (unsigned long long)s_hist[threadIdx.x]);
  }
  if (fin && last_block(&ctl->done) && threadIdx.x == 0)
    finalize_step<true>(*A.vol, ctl, A.ring, A.ring_cap, A.keys);
}

// Random init: sigma_a(c) = floor(w q / 2^32), w word c mod 4 of
// Philox((c / 4, 0, 0, 16 + a)); ordered init: every sigma 0.  The eta
// copies are written afterwards by k_eta_bits3.
__global__ void __launch_bounds__(kThreads3) k_init3(uint32_t* __restrict__ state, uint32_t N,
                                                      uint32_t groups, uint32_t q, int random,
                                                      RoundKeys K) {
  for (uint32_t gi = blockIdx.x * kThreads3 + threadIdx.x; gi < groups;
       gi += gridDim.x * kThreads3) {
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if (random) {
      for (int a = 0; a < 6; ++a) {
        const Words4 r = philox(gi, 0u, 0u, kTagInit0 + (uint32_t)a, K);
        const uint32_t rw[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] |= __umulhi(rw[i], q) << (4 * a);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (gi * 4u + (uint32_t)i < N) state[gi * 4u + (uint32_t)i] = w[i];
  }
}

// Full count of a lattice: N_HB_raw (arms 0, 2, 4 against arms 1, 3, 5 of
// the +x, +y, +z neighbours, on edges with eta = 1) and N_sigma (equal pairs
// among the six arms)
// added to acc2[0], acc2[1]; N_q' added to hist[0..8).  Either may be NULL.
__global__ void __launch_bounds__(kThreads3) k_count3(const uint32_t* __restrict__ state,
                                                       uint32_t L, uint32_t L2, uint32_t N,
                                                       FastDiv div_L, FastDiv div_L2,
                                                       unsigned long long* acc2,
                                                       unsigned long long* hist) {
  __shared__ unsigned long long s_cnt[8];
  if (threadIdx.x < 8) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  uint32_t hb = 0, pairs = 0, unused = 0;
  uint32_t h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (uint32_t c = blockIdx.x * kThreads3 + threadIdx.x; c < N; c += gridDim.x * kThreads3) {
    const uint32_t z = fdiv(c, div_L2);
    const uint32_t rem = c - z * L2;
    const uint32_t y = fdiv(rem, div_L);
    const uint32_t x = rem - y * L;
    const uint32_t w = state[c];
    const uint32_t wx = state[(x + 1u == L) ? c + 1u - L : c + 1u];
    const uint32_t wy = state[(y + 1u == L) ? c + L - L2 : c + L];
    const uint32_t wz = state[(z + 1u == L) ? c + L2 - N : c + L2];
    // a bond counts on an allowed edge only (the eta copy of the +axis arm)
    hb += (uint32_t)(((w >> 0) & 7u) == ((wx >> 4) & 7u)) & ((w >> 3) & 1u);
    hb += (uint32_t)(((w >> 8) & 7u) == ((wy >> 12) & 7u)) & ((w >> 11) & 1u);
    hb += (uint32_t)(((w >> 16) & 7u) == ((wz >> 20) & 7u)) & ((w >> 19) & 1u);
    const uint32_t cnt = count_word(w);
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const uint32_t m = (cnt >> (4 * v)) & 15u;
      pairs += m * (m - 1u) / 2u;
      h[v] += m;
    }
  }
  if (hist)
    for (int v = 0; v < 8; ++v)
      if (h[v]) atomicAdd(&s_cnt[v], (unsigned long long)h[v]);
  block_sum3<kThreads3>(hb, pairs, unused);
  if (threadIdx.x == 0 && acc2) {
    atomicAdd(&acc2[0], (unsigned long long)hb);
    atomicAdd(&acc2[1], (unsigned long long)pairs);
  }
  __syncthreads();
  if (hist && threadIdx.x < 8 && s_cnt[threadIdx.x]) atomicAdd(&hist[threadIdx.x], s_cnt[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// eta (App. A).  Cube (colour, X, Y, Z) has its corner of smallest
// coordinates at (2X + colour, 2Y + colour, 2Z + colour); corner j sits at
// offset (j & 1, (j >> 1) & 1, (j >> 2) & 1); edge e runs along axis d = e / 4
// from corner lo(e) -- the (e % 4)-th corner with bit d clear -- to lo(e) |
// (1 << d).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int edge_lo(int e) {
  const int d = e >> 2, k = e & 3;
  // corners with bit d clear, in increasing order: d = 0: 0 2 4 6; d = 1:
  // 0 1 4 5; d = 2: 0 1 2 3
  return (d == 0) ? 2 * k : (d == 1) ? ((k & 1) | ((k >> 1) << 2)) : k;
}

// The eight corner cells of a cube: the corner of smallest coordinates and
// the steps +x, +y, +z from it (periodic).
__device__ __forceinline__ void cube_corners(const Args3& A, uint32_t cube, uint32_t cell[8]) {
  const uint32_t H = A.H, H2 = H * H;
  const uint32_t colour = (cube >= H2 * H) ? 1u : 0u;
  const uint32_t rest = cube - colour * H2 * H;
  const uint32_t Zc = fdiv(rest, A.div_H);  // Z H + Y
  const uint32_t X = rest - Zc * H;
  const uint32_t Z = fdiv(Zc, A.div_H);
  const uint32_t Y = Zc - Z * H;
  const uint32_t L = A.L, L2 = A.L2;
  const uint32_t x0 = 2u * X + colour, y0 = 2u * Y + colour, z0 = 2u * Z + colour;
  const uint32_t base = z0 * L2 + y0 * L + x0;
  const uint32_t dx = (x0 + 1u == L) ? 1u - L : 1u;
  const uint32_t dy = (y0 + 1u == L) ? L - L2 : L;
  const uint32_t dz = (z0 + 1u == L) ? L2 - A.N : L2;  // unsigned wrap-around
  cell[0] = base;
  cell[1] = base + dx;
  cell[2] = base + dy;
  cell[3] = cell[1] + dy;
  cell[4] = base + dz;
  cell[5] = cell[1] + dz;
  cell[6] = cell[2] + dz;
  cell[7] = cell[3] + dz;
}

// The bonded edges of a cube (sigma only; eta is not read) in the packed
// layout of the edge masks: edge e = 4 d + k (axis d, k-th lower corner)
// at bit 8 k + 7 - d.  For axis d, byte d of a corner word holds its +d arm
// (low nibble) and -d arm (high nibble); the bytes of the four lower and of
// the four upper corners are gathered into one word each, and one nibble
// comparison per byte tests the four edges at once.
__device__ __forceinline__ uint32_t cube_bonds_packed(const uint32_t w[8]) {
  uint32_t bonds = 0;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    // corners with bit d clear, in increasing order, and their +d partners
    const int l0 = (d == 0) ? 0 : 0, l1 = (d == 0) ? 2 : 1, l2 = (d == 0) ? 4 : (d == 1) ? 4 : 2,
              l3 = (d == 0) ? 6 : (d == 1) ? 5 : 3;
    const int u = 1 << d;
    const uint32_t sel = (uint32_t)d | ((uint32_t)(4 + d) << 4);
    const uint32_t lo = __byte_perm(__byte_perm(w[l0], w[l1], sel), __byte_perm(w[l2], w[l3], sel),
                                    0x5410u);
    const uint32_t hi = __byte_perm(__byte_perm(w[l0 | u], w[l1 | u], sel),
                                    __byte_perm(w[l2 | u], w[l3 | u], sel), 0x5410u);
    // byte k: the +d arm of lower corner k against the -d arm of its partner
    const uint32_t m = (lo ^ (hi >> 4)) & 0x07070707u;
    const uint32_t differ = (m | 0x80808080u) - 0x01010101u;  // bit 7 set where m != 0
    bonds |= (~differ & 0x80808080u) >> d;
  }
  return bonds;
}

// An edge mask (bit e = edge e) in the packed layout of cube_bonds_packed.
__device__ __forceinline__ uint32_t pack_edge_mask(uint32_t m12) {
  uint32_t p = 0;
#pragma unroll
  for (int e = 0; e < 12; ++e) p |= ((m12 >> e) & 1u) << (8 * (e & 3) + 7 - (e >> 2));
  return p;
}

// The eta-copy flips of the corner words for the edges set in a packed flip
// mask: the +d arm (bit 8 d + 3) of the lower corner and the -d arm (bit
// 8 d + 7) of the upper corner of each edge.
__device__ __forceinline__ void cube_flip_bits(uint32_t flip, uint32_t x[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) x[j] = 0u;
#pragma unroll
  for (int e = 0; e < 12; ++e) {
    const int d = e >> 2, lo = edge_lo(e), hi = lo | (1 << d);
    const uint32_t f = (flip >> (8 * (e & 3) + 7 - d)) & 1u;
    x[lo] ^= f << (8 * d + 3);
    x[hi] ^= f << (8 * d + 7);
  }
}

// Step 2 of the MC step: one Metropolis move of every cube's configuration
// with the sigma fixed -- proposal (c + 1 + k) mod 9, k = floor(r0 8 / 2^32),
// accepted iff r1 < T[g][dN_HB + 4] with r = Philox((cube, step, 5)); the
// edges leaving the matching become allowed, those entering it forbidden,
// so dN_HB = |bonded & old| - |bonded & new|.  An accepted move rewrites the
// cube's byte and flips the eta copies of the changed edges in its corner
// words (atomic XOR: the other cube of each corner may flip other bits of
// the same word at the same time); the changes of N_HB_raw go to the step's
// accumulator.
__global__ void __launch_bounds__(kThreads3) k_eta3(Args3 A) {
  __shared__ unsigned long long sT[9];
  __shared__ uint32_t sMask[9];
  __shared__ int red[kThreads3 / 32];
  Ctrl* ctl = A.ctrl;
  const int g = ctl->next_g;
  const long long step = ctl->sweep;
  if (threadIdx.x < 9) {
    sT[threadIdx.x] = A.eta_table[g * 9 + threadIdx.x];
    sMask[threadIdx.x] = pack_edge_mask(A.masks[threadIdx.x]);
  }
  __syncthreads();
  const uint32_t s_lo = (uint32_t)((unsigned long long)step & 0xFFFFFFFFu);
  const uint32_t s_hi = (uint32_t)((unsigned long long)step >> 32);
  int dsum = 0;
  for (uint32_t cube = blockIdx.x * kThreads3 + threadIdx.x; cube < A.ncube;
       cube += gridDim.x * kThreads3) {
    uint32_t cell[8], w[8];
    cube_corners(A, cube, cell);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      w[j] = dcheck(cell[j] < A.N, &ctl->error, kSiteEta3) ? A.state[cell[j]] : 0u;
    const uint32_t bonds = cube_bonds_packed(w);
    const uint32_t old = A.eta[cube];
    const Words4 r = philox(cube, s_lo, s_hi, kTagEta, A.keys);
    uint32_t nw = old + 1u + __umulhi(r.x, 8u);
    if (nw >= 9u) nw -= 9u;
    if (!dcheck(old < 9u, &ctl->error, kSiteEta3)) continue;
    const uint32_t zo = sMask[old], zn = sMask[nw];
    const int dhb = __popc(bonds & zo) - __popc(bonds & zn);
    if ((unsigned long long)r.y < sT[dhb + 4]) {
      A.eta[cube] = (uint8_t)nw;
      dsum += dhb;
      uint32_t x[8];
      cube_flip_bits(zo ^ zn, x);
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (x[j]) atomicXor(&A.state[cell[j]], x[j]);
    }
  }
  // block sum of the changes of N_HB_raw, one atomic per block
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xFFFFFFFFu, dsum, o);
  if ((threadIdx.x & 31u) == 0u) red[threadIdx.x >> 5] = dsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int i = 0; i < kThreads3 / 32; ++i) t += red[i];
    if (t) atomicAdd(&ctl->acc_hb, (unsigned long long)(long long)t);
  }
}

// Initial cube configurations: floor(r0 9 / 2^32) with r = Philox((cube, 0,
// 0, 6)) (random init) or 0 (ordered init).
__global__ void __launch_bounds__(kThreads3) k_eta_init3(uint8_t* eta, uint32_t ncube, int random,
                                                          RoundKeys K) {
  for (uint32_t cube = blockIdx.x * kThreads3 + threadIdx.x; cube < ncube;
       cube += gridDim.x * kThreads3) {
    uint32_t cfg = 0;
    if (random) cfg = __umulhi(philox(cube, 0u, 0u, kTagEtaInit, K).x, 9u);
    eta[cube] = (uint8_t)cfg;
  }
}

// The eta copies of every cell word from the cube configurations (all 1
// without eta moves).  The edge of arm a of cell (x, y, z) joins v and v +
// e_d (d = a / 2; v is the cell for a +d arm, its -d neighbour otherwise);
// its cube has v's coordinate along d and, along each other axis u, v_u or
// v_u - 1, whichever has the parity of v_d; the edge's number follows from
// v's corner in that cube.
__global__ void __launch_bounds__(kThreads3) k_eta_bits3(Args3 A) {
  for (uint32_t c = blockIdx.x * kThreads3 + threadIdx.x; c < A.N; c += gridDim.x * kThreads3) {
    const uint32_t L = A.L;
    const uint32_t z = fdiv(c, A.div_L2);
    const uint32_t rem = c - z * A.L2;
    const uint32_t y = fdiv(rem, A.div_L);
    const uint32_t x = rem - y * L;
    uint32_t bits = kEtaBits;
    if (A.eta) {
      bits = 0u;
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const int d = a >> 1;
        uint32_t v[3] = {x, y, z};
        if (a & 1) v[d] = (v[d] == 0u) ? L - 1u : v[d] - 1u;
        uint32_t cc[3];
        int j = 0;
#pragma unroll
        for (int u = 0; u < 3; ++u) {
          if (u == d || ((v[u] ^ v[d]) & 1u) == 0u) {
            cc[u] = v[u];
          } else {
            cc[u] = (v[u] == 0u) ? L - 1u : v[u] - 1u;
            j |= 1 << u;
          }
        }
        const uint32_t colour = v[d] & 1u;
        const uint32_t cube = ((colour * A.H + (cc[2] >> 1)) * A.H + (cc[1] >> 1)) * A.H + (cc[0] >> 1);
        // rank of corner j among the corners with bit d clear
        const int k = (d == 0) ? (j >> 1) : (d == 1) ? ((j & 1) | ((j >> 2) << 1)) : j;
        const int e = 4 * d + k;
        uint32_t cfg = 0u;
        if (dcheck(cube < A.ncube, &A.ctrl->error, kSiteEta3)) cfg = A.eta[cube];
        const uint32_t forbidden = (cfg < 9u) ? ((uint32_t)A.masks[cfg] >> e) & 1u : 0u;
        bits |= (forbidden ^ 1u) << (4 * a + 3);
      }
    }
    A.state[c] = (A.state[c] & kArmBits) | bits;
  }
}

// ---------------------------------------------------------------------------
// Small cubes resident in one thread-block cluster of nct = 8 or 16 CTAs (L a
// multiple of nct, 16 <= L <= 64): CTA r holds the z-planes [r R, (r+1) R),
// R = L / nct, in shared memory for every step of a call.  The step's
// launches of k_pass3 become segments separated by cluster barriers; the
// z-partners across a slab boundary are read from the neighbouring CTA's
// shared memory.  Every cell is updated with the same draws and rule as in
// k_pass3, so the results are identical.  A 33rd warp in CTA 0 decides the
// next step's volume move, overlapping the first segment; CTA 0 commits the
// step after the last segment.  All CTAs follow the same plan (computed from
// the step by each), so they meet the same barriers.
// ---------------------------------------------------------------------------
constexpr int kRes3Ctas = 8;
constexpr int kRes3Threads = 256;
constexpr int kRes3Block = kRes3Threads + 64;  // + two volume warps
constexpr int kRes3MaxSide = 64;
// the automatic choice takes the resident form up to this side (measured
// per MC step with the eta update, resident against four launches: 16^3 7.6
// against 14.6 us, 24^3 9.3 against 15.3, 32^3 12.1 against 16.1 with a
// 16-CTA cluster (19.7 with 8); beyond, 16 SMs do too much of the work:
// 48^3 31.5 against 16.2, 64^3 66.7 against 17.7)
constexpr int kRes3AutoSide = 32;

__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait;" ::: "memory"); }
__device__ __forceinline__ void cl_barrier() {
  cl_arrive();
  cl_wait();
}
__device__ __forceinline__ void sweepers3_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kRes3Threads) : "memory");
}

template <bool CMP64>
__global__ void __launch_bounds__(kRes3Block) k_resident3(Args3 A, long long n_steps) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ uint32_t cube[];  // planes z0 .. z0 + R - 1, L^2 words each
  __shared__ Row3 sRows[33];
  __shared__ uint32_t sProp[64];
  __shared__ unsigned long long sT64[CMP64 ? 33 : 1];
  __shared__ unsigned long long s_acc[3];   // CTA 0: the step's dN_HB, dN_sigma, moves
  __shared__ unsigned long long s_hist[8];  // CTA 0: N_q' of a recorded step
  __shared__ uint32_t s_h[8];               // this CTA's N_q' of a recorded step
  __shared__ uint32_t red[3][kRes3Threads / 32];
  __shared__ int s_next_g, s_plan;
  __shared__ VolumeArgs sV;
  __shared__ double s_xch;
  __shared__ unsigned long long sEtaT[18];  // eta move thresholds [g][dN_HB + 4]
  __shared__ uint32_t sEtaMask[9];          // edge masks of the nine cube configurations
  // CTA 0 keeps the lattice's scalar state in shared memory for the whole
  // call and writes it back at the end (no global round trip per step)
  __shared__ Ctrl s_ctl;
  Ctrl* const gctl = A.ctrl;
  const int nct = (int)cluster.num_blocks();  // 8, or 16 for cubes with L a multiple of 16
  const uint32_t L = A.L, L2 = A.L2, G = A.G, R = L / (uint32_t)nct, z0 = rank * R;
  const bool eta_on = A.eta != nullptr;  // the eta step (App. A) opens every step
  const uint32_t q = A.q, qm1 = q - 1u;
  const bool sweeper = threadIdx.x < kRes3Threads;
  const long long step0 = gctl->sweep;
  const int every = gctl->record_every;
  if (rank == 0 && threadIdx.x == 0) s_ctl = *gctl;
  Ctrl* const ctl = &s_ctl;  // meaningful in CTA 0 only
  uint32_t* const st = A.state;

  for (uint32_t i = threadIdx.x; i < R * L2; i += blockDim.x) cube[i] = st[z0 * L2 + i];
  if (threadIdx.x >= 64 && threadIdx.x < 128) {
    const uint32_t sgm = (threadIdx.x - 64) >> 3, k = (threadIdx.x - 64) & 7u;
    uint32_t sp = sgm + 1u + k;
    while (sp >= q) sp -= q;
    sProp[threadIdx.x - 64] = (sgm < q && k + 1u < q) ? sp * kR7 : 0u;
  }
  stage_volume_args(&sV, A.vol);
  if (eta_on && threadIdx.x < 18) sEtaT[threadIdx.x] = A.eta_table[threadIdx.x];
  if (eta_on && threadIdx.x < 9) sEtaMask[threadIdx.x] = pack_edge_mask(A.masks[threadIdx.x]);
  if (rank == 0 && threadIdx.x == 0) s_next_g = ctl->next_g;
  // the planes just below and above this slab, in the neighbours' shared memory
  const uint32_t* below = cluster.map_shared_rank(cube, (rank + nct - 1) % nct) + (R - 1) * L2;
  const uint32_t* above = cluster.map_shared_rank(cube, (rank + 1) % nct);
  unsigned long long* acc0 = cluster.map_shared_rank(&s_acc[0], 0);
  unsigned long long* hist0 = cluster.map_shared_rank(&s_hist[0], 0);
  const int* next_g0 = cluster.map_shared_rank(&s_next_g, 0);
  int g_cur = -1;
  __syncthreads();
  cl_barrier();

  for (long long it = 0; it < n_steps; ++it) {
    const long long step = step0 + it;
    if (threadIdx.x == 0) s_plan = (int)make_plan(step, A.keys);
    __syncthreads();
    const uint32_t plan = (uint32_t)s_plan;
    const int nseg = plan_launches(plan);
    const bool rec = step_recorded(every, step);
    if (!sweeper) {
      // the end of the eta segment (with eta moves), else of segment 0
      cl_arrive();
      if (rank == 0) {  // the two volume warps: the move on two FP64 pipes
        VolumeResult r;
        const bool ok = volume_decide_pair<3>((int)((threadIdx.x - kRes3Threads) >> 5), sV,
                                              step + 1, ctl->next_V, ctl->next_u, ctl->next_g,
                                              -1, A.keys, &r, &s_xch);
        if (threadIdx.x == kRes3Threads && ok) {
          ctl->ahead_V = r.V;
          ctl->ahead_u = r.u;
          ctl->ahead_g = r.g;
          ctl->ahead_acc = r.accepted;
          ctl->ahead_state = 1;
        }
      }
      __syncwarp();
      cl_wait();
      for (int j = eta_on ? 0 : 1; j < nseg; ++j) cl_barrier();  // the later segments
      cl_barrier();                                              // the step committed
      continue;
    }
    const int g = *next_g0;
    if (g != g_cur) {  // uniform over the CTA's sweepers
      if (threadIdx.x < 33) {
        const unsigned long long t = A.table[g * 33 + threadIdx.x];
        if (CMP64) sT64[threadIdx.x] = t;
        const int dhb = (int)threadIdx.x / 11 - 1, dc = (int)threadIdx.x % 11 - 5;
        sRows[threadIdx.x].t = (uint32_t)(t - 1ull);
        sRows[threadIdx.x].delta = (1u << 24) + ((uint32_t)(dhb + 1) << 16) + (uint32_t)(dc + 5);
      }
      g_cur = g;
    }
    if (rank == 0 && threadIdx.x < 3) s_acc[threadIdx.x] = 0;
    if (rank == 0 && threadIdx.x < 8) s_hist[threadIdx.x] = 0;
    if (threadIdx.x < 8) s_h[threadIdx.x] = 0;
    sweepers3_sync();
    const uint32_t s_lo = (uint32_t)((unsigned long long)step & 0xFFFFFFFFu);
    const uint32_t s_hi = (uint32_t)((unsigned long long)step >> 32);
    uint32_t nacc = 0, hb_b = 0, dc_b = 0, pk = 0;
    int eta_dhb = 0;  // this thread's changes of N_HB_raw by accepted cube moves
    if (eta_on) {
      // Step 2 of the MC step, as k_eta3: one Metropolis move of every
      // checkerboard cube whose lower z-plane lies in this slab (its upper
      // plane may be the next CTA's first: distributed shared memory); the
      // eta copies of a changed edge are flipped by atomic XOR in the two
      // corner words (other cubes flip other bits of the same words).
      const uint32_t H = A.H;
      uint32_t zmin[2], zcnt[2];
#pragma unroll
      for (uint32_t c = 0; c < 2u; ++c) {
        const uint32_t lo = (z0 + 1u - c) >> 1;                // first Z with 2Z + c >= z0
        const uint32_t hi = min((z0 + R + 1u - c) >> 1, H);    // first Z with 2Z + c >= z0 + R
        zmin[c] = lo;
        zcnt[c] = (hi > lo) ? hi - lo : 0u;
      }
      const uint32_t HH = H * H, n0 = zcnt[0] * HH, ncub = n0 + zcnt[1] * HH;
      for (uint32_t i = threadIdx.x; i < ncub; i += kRes3Threads) {
        const uint32_t c = (i >= n0) ? 1u : 0u;
        const uint32_t k = i - c * n0;
        const uint32_t zy = k / H, X = k - zy * H;
        const uint32_t Zr = zy / H, Y = zy - Zr * H;
        const uint32_t Z = zmin[c] + Zr;
        const uint32_t cb = c * HH * H + (Z * H + Y) * H + X;  // global cube index
        const uint32_t zl = 2u * Z + c - z0;                    // local plane of the lower corners
        const uint32_t x0 = 2u * X + c, y0 = 2u * Y + c;
        const uint32_t x1 = (x0 + 1u == L) ? 0u : x0 + 1u, y1 = (y0 + 1u == L) ? 0u : y0 + 1u;
        uint32_t* const plo = cube + zl * L2;
        uint32_t* const phi = (zl + 1u < R) ? cube + (zl + 1u) * L2 : const_cast<uint32_t*>(above);
        uint32_t* wp[8];
        uint32_t w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          wp[j] = ((j & 4) ? phi : plo) + ((j & 2) ? y1 : y0) * L + ((j & 1) ? x1 : x0);
          w[j] = dcheck(zl < R && cb < A.ncube, &gctl->error, kSiteResident3) ? *wp[j] : 0u;
        }
        const uint32_t bonds = cube_bonds_packed(w);
        const uint32_t old = A.eta[cb];
        if (!dcheck(old < 9u, &gctl->error, kSiteResident3)) continue;
        const Words4 r = philox(cb, s_lo, s_hi, kTagEta, A.keys);
        uint32_t nw = old + 1u + __umulhi(r.x, 8u);
        if (nw >= 9u) nw -= 9u;
        const uint32_t zo = sEtaMask[old], zn = sEtaMask[nw];
        const int dhb = __popc(bonds & zo) - __popc(bonds & zn);
        if ((unsigned long long)r.y < sEtaT[g * 9 + dhb + 4]) {
          A.eta[cb] = (uint8_t)nw;
          eta_dhb += dhb;
          uint32_t x[8];
          cube_flip_bits(zo ^ zn, x);
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (x[j]) atomicXor(wp[j], x[j]);
        }
      }
      cl_barrier();  // every flip is in place before the sigma passes
    }
    for (int j = 0; j < nseg; ++j) {
      int arms[3] = {0, 0, 0};
      const int n_arms = plan_arms(plan, j, arms);
      // loads of the slab's words (and the neighbouring slabs' planes),
      // index-checked in debug builds
      const uint32_t slab = R * L2;
      auto vec = [&](const uint32_t* base, uint32_t idx, uint32_t n) -> uint4 {
        return dcheck((idx & 3u) == 0u && idx + 3u < n, &gctl->error, kSiteResident3)
                   ? *reinterpret_cast<const uint4*>(base + idx)
                   : make_uint4(0u, 0u, 0u, 0u);
      };
      auto word = [&](uint32_t idx) -> uint32_t {
        return dcheck(idx < slab, &gctl->error, kSiteResident3) ? cube[idx] : 0u;
      };
      for (uint32_t i = threadIdx.x; i < R * L2 / 4u; i += kRes3Threads) {
        const uint32_t c0 = 4u * i;  // local cell of the group
        const uint32_t zl = c0 / L2, rem = c0 - zl * L2, y = rem / L, xg = (rem - y * L) >> 2;
        const uint32_t gi = (z0 * L2 + c0) >> 2;  // global group index (Philox counter)
        const uint4 own = vec(cube, c0, slab);
        uint32_t w0 = own.x, w1 = own.y, w2 = own.z, w3 = own.w;
        for (int p = 0; p < n_arms; ++p) {
          const int a = arms[p];
          uint4 nb;
          if (a == 0) {
            nb = make_uint4(own.y, own.z, own.w, word((xg + 1u == G) ? c0 + 4u - L : c0 + 4u));
          } else if (a == 1) {
            nb = make_uint4(word((xg == 0u) ? c0 + L - 1u : c0 - 1u), own.x, own.y, own.z);
          } else if (a == 2) {
            nb = vec(cube, (y == L - 1u) ? c0 + L - L2 : c0 + L, slab);
          } else if (a == 3) {
            nb = vec(cube, (y == 0u) ? c0 + L2 - L : c0 - L, slab);
          } else if (a == 4) {
            nb = (zl == R - 1u) ? vec(above, rem, L2) : vec(cube, c0 + L2, slab);
          } else {
            nb = (zl == 0u) ? vec(below, rem, L2) : vec(cube, c0 - L2, slab);
          }
          const uint32_t sh = 4u * (uint32_t)a, nsh = 24u - 4u * (uint32_t)(a ^ 1);
          const uint32_t amask = 0xFu << sh;
          const Words4 r = philox(gi, s_lo, s_hi, kTagArm0 + (uint32_t)a, A.keys);
          w0 = update_arm3<CMP64>(w0, nb.x, r.x, sh, nsh, amask, qm1, sProp, sRows, sT64, pk);
          w1 = update_arm3<CMP64>(w1, nb.y, r.y, sh, nsh, amask, qm1, sProp, sRows, sT64, pk);
          w2 = update_arm3<CMP64>(w2, nb.z, r.z, sh, nsh, amask, qm1, sProp, sRows, sT64, pk);
          w3 = update_arm3<CMP64>(w3, nb.w, r.w, sh, nsh, amask, qm1, sProp, sRows, sT64, pk);
        }
        unpack_counts(pk, nacc, hb_b, dc_b);
        if (dcheck(c0 + 3u < slab, &gctl->error, kSiteResident3))
          *reinterpret_cast<uint4*>(cube + c0) = make_uint4(w0, w1, w2, w3);
        if (rec && j == nseg - 1) hist_group(w0, w1, w2, w3, s_h);
      }
      if (j == nseg - 1) {
        // the step's counts (and N_q') into CTA 0 before the last barrier
        uint32_t a1 = hb_b - nacc + (uint32_t)eta_dhb, a2 = dc_b - 5u * nacc, a3 = nacc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          a1 += __shfl_xor_sync(0xFFFFFFFFu, a1, o);
          a2 += __shfl_xor_sync(0xFFFFFFFFu, a2, o);
          a3 += __shfl_xor_sync(0xFFFFFFFFu, a3, o);
        }
        if ((threadIdx.x & 31) == 0) {
          red[0][threadIdx.x >> 5] = a1;
          red[1][threadIdx.x >> 5] = a2;
          red[2][threadIdx.x >> 5] = a3;
        }
        sweepers3_sync();
        if (threadIdx.x == 0) {
          a1 = a2 = a3 = 0;
          for (int w = 0; w < kRes3Threads / 32; ++w) {
            a1 += red[0][w];
            a2 += red[1][w];
            a3 += red[2][w];
          }
          atomicAdd(&acc0[0], (unsigned long long)(long long)(int)a1);
          atomicAdd(&acc0[1], (unsigned long long)(long long)(int)a2);
          atomicAdd(&acc0[2], (unsigned long long)a3);
        }
        if (rec && threadIdx.x < 8 && s_h[threadIdx.x])
          atomicAdd(&hist0[threadIdx.x], (unsigned long long)s_h[threadIdx.x]);
      }
      cl_barrier();  // segment j done in every CTA
    }
    if (rank == 0 && threadIdx.x == 0) {
      ctl->acc_hb = s_acc[0];
      ctl->acc_pairs = s_acc[1];
      ctl->acc_moves = s_acc[2];
      if (rec)
        for (int v = 0; v < 8; ++v) ctl->acc_hist[v] = s_hist[v];
      finalize_step<true>(sV, ctl, A.ring, A.ring_cap, A.keys);
      s_next_g = ctl->next_g;
    }
    cl_barrier();  // the step committed
  }
  // CTA 0's scalar state back to the handle (every CTA is past its last
  // index check, so the device error word is final)
  if (rank == 0 && threadIdx.x == 0) {
    s_ctl.error = *(volatile unsigned int*)&gctl->error;
    *gctl = s_ctl;
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < R * L2; i += blockDim.x) st[z0 * L2 + i] = cube[i];
}

// Observables of the committed state with N_q' from a count of the lattice.
__global__ void k_observables3(const VolumeArgs* __restrict__ V, const Ctrl* ctl,
                               const unsigned long long* hist, cvf_obs* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    cvf_obs o = make_obs(*V, ctl);
    for (int v = 0; v < 8; ++v) o.n_state[v] = (long long)hist[v];
    *out = o;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

template <bool CMP64>
cudaError_t launch_resident3_t(const Args3& A, int nct, long long n_steps, cudaStream_t s,
                               bool query, int* clusters) {
  const void* fn = (const void*)k_resident3<CMP64>;
  const size_t smem = (size_t)(A.L / nct) * A.L2 * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(nct);
  cfg.blockDim = dim3(kRes3Block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = nct;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (query) return cudaOccupancyMaxActiveClusters(clusters, fn, &cfg);
  return cudaLaunchKernelEx(&cfg, k_resident3<CMP64>, A, n_steps);
}

int query_clusters3(const Args3& A, bool cmp64, int nct) {
  int clusters = 0;
  const cudaError_t e = cmp64 ? launch_resident3_t<true>(A, nct, 0, nullptr, true, &clusters)
                              : launch_resident3_t<false>(A, nct, 0, nullptr, true, &clusters);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return clusters;
}

// CTAs of the resident cluster: 16 (a non-portable cluster size) where the
// side splits into 16 slabs of at least two planes and the GPU can place
// such a cluster, else 8.  At 32^3 the 16-CTA form takes 12.1 us per MC step
// against 19.7 us with 8 CTAs (48^3: 31.5 / 57.9, 64^3: 66.7 / 127.4).
int resident3_ctas(const Args3& A, bool cmp64) {
  if (A.L % 16u == 0u && A.L >= 32u && query_clusters3(A, cmp64, 16) >= 1) return 16;
  return kRes3Ctas;
}

cudaError_t launch_resident3(const Args3& A, bool cmp64, int nct, long long n_steps,
                             cudaStream_t s) {
  return cmp64 ? launch_resident3_t<true>(A, nct, n_steps, s, false, nullptr)
               : launch_resident3_t<false>(A, nct, n_steps, s, false, nullptr);
}

// Whether the cube can run resident in one cluster on this GPU.
bool resident3_fits(const Args3& A, bool cmp64) {
  if (A.L % kRes3Ctas != 0 || A.L < 2 * kRes3Ctas || (int)A.L > kRes3MaxSide) return false;
  return query_clusters3(A, cmp64, kRes3Ctas) >= 1;
}

// The automatic choice: resident up to 24^3 with any cluster, and at 32^3
// only when the 16-CTA cluster fits (with 8 CTAs it is slower there than
// the launch form).
bool resident3_auto(const Args3& A, bool cmp64) {
  if ((int)A.L > kRes3AutoSide || !resident3_fits(A, cmp64)) return false;
  return (int)A.L <= 24 || resident3_ctas(A, cmp64) == 16;
}

int check_params3(const cvf_params* p) {
  if (!p) return set_error(CVF_EINVAL, "params is NULL");
  if (p->L < 2 || p->L > kMaxSide3)
    return set_error(CVF_EINVAL, "L=%d: need 2 <= L <= %d for the cubic lattice", p->L,
                     kMaxSide3);
  if (p->schedule != CVF_SCHED_LAYERED)
    return set_error(CVF_EINVAL, "the cubic lattice runs the layered schedule only");
  if (p->rng_words != 1)
    return set_error(CVF_EINVAL, "the cubic lattice draws one word per update (rng_words 1)");
  if (p->eta_moves != 0 && p->eta_moves != 1)
    return set_error(CVF_EINVAL, "eta_moves=%d must be 0 or 1", p->eta_moves);
  if (p->eta_moves && (p->L & 1))
    return set_error(CVF_EINVAL, "L=%d: the eta update of the checkerboard cubes needs an even L",
                     p->L);
  cvf_params t = *p;
  t.L = 2;          // the side rules of the square lattice do not apply here
  t.eta_moves = 0;  // nor its eta rule
  return check_params(&t);
}

// The nine configurations of a checkerboard cube: the 12-bit masks of the
// perfect matchings of the cube graph (four edges covering each corner
// once), in increasing order; edge e runs along axis e / 4 from the (e %
// 4)-th corner with that axis's bit clear.
void cube_matchings(uint16_t out[9]) {
  int n = 0;
  for (uint32_t m = 0; m < 4096u && n < 9; ++m) {
    if (__builtin_popcount(m) != 4) continue;
    int cover[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int e = 0; e < 12; ++e) {
      if (!((m >> e) & 1u)) continue;
      const int d = e / 4, k = e % 4;
      int lo = -1, seen = 0;
      for (int j = 0; j < 8 && lo < 0; ++j)
        if (!((j >> d) & 1) && seen++ == k) lo = j;
      cover[lo] += 1;
      cover[lo | (1 << d)] += 1;
    }
    bool ok = true;
    for (int j = 0; j < 8; ++j) ok = ok && cover[j] == 1;
    if (ok) out[n++] = (uint16_t)m;
  }
}

// Thresholds of a cube move [g][dN_HB + 4]: dH = -g J_eff dN_HB, T = 2^32
// when dH <= 0, else floor(exp(-dH/kT) 2^32).
void eta_table3(const cvf_params* p, unsigned long long out[18]) {
  const double J_eff = p->J - p->P * p->v_HB;
  for (int g = 0; g < 2; ++g)
    for (int i = 0; i < 9; ++i) {
      const double dH = -((double)g * J_eff) * (double)(i - 4);
      out[g * 9 + i] = (dH <= 0.0) ? (1ull << 32)
                                   : (unsigned long long)(std::exp(-dH / p->kT) * 4294967296.0);
    }
}

void threshold_table3(const cvf_params* p, uint64_t out[66]) {
  const double J_eff = p->J - p->P * p->v_HB;
  for (int g = 0; g < 2; ++g)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 11; ++j) {
        const int dhb = i - 1, dc = j - 5;
        const double dH = -((double)g * J_eff) * (double)dhb - p->J_sigma * (double)dc;
        out[(g * 3 + i) * 11 + j] = (dH <= 0.0)
                                        ? ((uint64_t)1 << 32)
                                        : (uint64_t)(std::exp(-dH / p->kT) * 4294967296.0);
      }
}

// Shells of the cubic lattice inside the cutoff: |d|^2 (ascending) and the
// number of lattice vectors of each length.
void cubic_shells(double cutoff, std::vector<int64_t>* d2, std::vector<int64_t>* mult) {
  d2->clear();
  mult->clear();
  const int R = (int)std::ceil(cutoff);
  std::vector<int64_t> count((size_t)3 * R * R + 1, 0);
  for (int i = -R; i <= R; ++i)
    for (int j = -R; j <= R; ++j)
      for (int k = -R; k <= R; ++k) {
        const int64_t s = (int64_t)i * i + (int64_t)j * j + (int64_t)k * k;
        if (s > 0) count[(size_t)s] += 1;
      }
  for (size_t s = 1; s < count.size(); ++s)
    if (count[s] > 0 && (double)s < cutoff * cutoff) {
      d2->push_back((int64_t)s);
      mult->push_back(count[s]);
    }
}

// FP64 parameters of the volume move for the cubic lattice: shell keys
// |d|^6 against cutoff^6, prefix sums of m/|d|^12 and m/|d|^6 in increasing
// |d|.
void fill_volume_args3(const cvf_params* p, long long N, const std::vector<int64_t>& d2,
                       const std::vector<int64_t>& mult, VolumeArgs* va) {
  std::memset(va, 0, sizeof(*va));
  va->N = N;
  va->epsilon = p->epsilon;
  const double c = p->cutoff;
  va->cutoff2 = c * c * c * c * c * c;
  va->J = p->J;
  va->J_sigma = p->J_sigma;
  va->v_HB = p->v_HB;
  va->kT = p->kT;
  va->P = p->P;
  va->dV_max = p->dv_max_frac * ((double)N * p->v_iso_init);
  va->volume_moves = p->volume_moves;
  va->dim = 3;
  va->nshell = (int32_t)d2.size();
  va->S12[0] = 0.0;
  va->S6[0] = 0.0;
  for (size_t s = 0; s < d2.size(); ++s) {
    const int64_t d6 = d2[s] * d2[s] * d2[s];
    va->shell_d2[s] = (double)d6;
    va->S12[s + 1] = va->S12[s] + (double)mult[s] / ((double)d6 * (double)d6);
    va->S6[s + 1] = va->S6[s] + (double)mult[s] / (double)d6;
  }
}

}  // namespace
}  // namespace cvf

using namespace cvf;

struct cvf3_handle {
  cvf_params p;
  long long N;
  cudaStream_t stream;
  cudaStream_t cap_stream;
  uint32_t* state;
  bool own_state;
  Ctrl* ctrl;
  cvf_obs* ring;
  long long ring_cap;
  long long ring_tail;
  cvf_obs* obs_dev;
  unsigned long long* table_dev;
  VolumeArgs* vol_dev;
  unsigned long long* rc_dev;  // 10 counters: N_q'[8], N_HB_raw, N_sigma
  uint8_t* eta;                // cube configurations (eta moves only)
  unsigned long long* eta_table_dev;
  void* host_pinned;
  Args3 args;
  bool cmp64;
  bool aligned;
  bool resident;  // the cube stays in one cluster's shared memory during a call
  int res_ctas;   // CTAs of that cluster (0 until it is first needed)
  int grid;
  int grid_count;
  int grid_eta;
  cudaGraphExec_t graph;
};

namespace {

void release3(cvf3_handle* h) {
  if (!h) return;
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->own_state && h->state) cudaFree(h->state);
  if (h->ctrl) cudaFree(h->ctrl);
  if (h->ring) cudaFree(h->ring);
  if (h->obs_dev) cudaFree(h->obs_dev);
  if (h->table_dev) cudaFree(h->table_dev);
  if (h->vol_dev) cudaFree(h->vol_dev);
  if (h->rc_dev) cudaFree(h->rc_dev);
  if (h->eta) cudaFree(h->eta);
  if (h->eta_table_dev) cudaFree(h->eta_table_dev);
  if (h->host_pinned) cudaFreeHost(h->host_pinned);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

const void* pass_kernel(bool aligned, bool cmp64) {
  if (aligned) return cmp64 ? (const void*)k_pass3<true, true> : (const void*)k_pass3<true, false>;
  return cmp64 ? (const void*)k_pass3<false, true> : (const void*)k_pass3<false, false>;
}

void enqueue_step3(cvf3_handle* h, cudaStream_t s) {
  if (h->eta) k_eta3<<<h->grid_eta, kThreads3, 0, s>>>(h->args);  // step 2: eta
  for (int j = 0; j < kLaunches3; ++j) {
    const int grid = h->grid + (j == 0 ? 1 : 0);
    if (h->aligned) {
      if (h->cmp64)
        k_pass3<true, true><<<grid, kThreads3, 0, s>>>(h->args, j);
      else
        k_pass3<true, false><<<grid, kThreads3, 0, s>>>(h->args, j);
    } else {
      if (h->cmp64)
        k_pass3<false, true><<<grid, kThreads3, 0, s>>>(h->args, j);
      else
        k_pass3<false, false><<<grid, kThreads3, 0, s>>>(h->args, j);
    }
  }
}

int build_graph3(cvf3_handle* h) {
  if (h->graph) return CVF_OK;
  cudaGraph_t g = nullptr;
  CVF_CUDA_CHECK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < kGraphSteps3; ++i) enqueue_step3(h, h->cap_stream);
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (e != cudaSuccess) return set_error(CVF_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->graph = nullptr;
    return set_error(CVF_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  return CVF_OK;
}

// Count the lattice into the control block (committed N_HB_raw, N_sigma) and
// prepare the next volume move; the cell words' eta copies are rewritten
// from the cube configurations first.
int recount_into_ctrl3(cvf3_handle* h) {
  static_assert(offsetof(Ctrl, acc_pairs) == offsetof(Ctrl, acc_hb) + 8, "layout");
  k_eta_bits3<<<h->grid_count, kThreads3, 0, h->stream>>>(h->args);
  k_count3<<<h->grid_count, kThreads3, 0, h->stream>>>(h->state, h->args.L, h->args.L2,
                                                        h->args.N, h->args.div_L, h->args.div_L2,
                                                        &h->ctrl->acc_hb, nullptr);
  k_commit_counts<<<1, 32, 0, h->stream>>>(h->ctrl);
  k_volume_prologue<<<1, 32, 0, h->stream>>>(h->vol_dev, h->ctrl, h->args.keys);
  CVF_CUDA_CHECK(cudaGetLastError());
  return CVF_OK;
}

}  // namespace

extern "C" {

int cvf3_params_physical(double T_kelvin, double P_MPa, cvf_params* out) {
  const int rc = cvf_params_physical(T_kelvin, P_MPa, out);
  if (rc) return rc;
  out->L = 16;
  out->v_iso_init = std::sqrt(2.0);
  out->schedule = CVF_SCHED_LAYERED;
  out->rng_words = 1;
  out->eta_moves = 1;
  return CVF_OK;
}

int cvf3_threshold_table(const cvf_params* p, uint64_t out[66]) {
  if (!out) return set_error(CVF_EINVAL, "out is NULL");
  const int rc = check_params3(p);
  if (rc) return rc;
  threshold_table3(p, out);
  return CVF_OK;
}

int cvf3_create(const cvf_params* p, void* stream, void* dev_state, cvf3_handle** out) {
  NvtxRange nvtx_range("cvf3_create");
  if (!out) return set_error(CVF_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = check_params3(p);
  if (rc) return rc;
  if (dev_state && (reinterpret_cast<uintptr_t>(dev_state) & 15u))
    return set_error(CVF_EINVAL, "dev_state must be 16-byte aligned");
  std::vector<int64_t> d2, mult;
  cubic_shells(p->cutoff, &d2, &mult);
  if ((int)d2.size() > kMaxShells)
    return set_error(CVF_EINVAL, "cutoff %g needs %zu shells (max %d)", p->cutoff, d2.size(),
                     kMaxShells);
  cvf3_handle* h = new (std::nothrow) cvf3_handle();
  if (!h) return set_error(CVF_ENOMEM, "host allocation failed");
  std::memset(h, 0, sizeof(*h));
  h->p = *p;
  const uint32_t L = (uint32_t)p->L;
  h->N = (long long)L * L * L;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->ring_cap = kRingCap3;
#define CREATE_CHECK(expr)                                                        \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      int code_ = (e_ == cudaErrorMemoryAllocation) ? CVF_ENOMEM : CVF_ECUDA;     \
      set_error(code_, "%s failed: %s", #expr, cudaGetErrorString(e_));           \
      release3(h);                                                                \
      return code_;                                                               \
    }                                                                             \
  } while (0)
  CREATE_CHECK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  if (dev_state) {
    h->state = reinterpret_cast<uint32_t*>(dev_state);
    h->own_state = false;
  } else {
    CREATE_CHECK(cudaMalloc(&h->state, sizeof(uint32_t) * (size_t)h->N));
    h->own_state = true;
  }
  CREATE_CHECK(cudaMalloc(&h->ctrl, sizeof(Ctrl)));
  CREATE_CHECK(cudaMalloc(&h->ring, sizeof(cvf_obs) * (size_t)h->ring_cap));
  CREATE_CHECK(cudaMalloc(&h->obs_dev, sizeof(cvf_obs)));
  CREATE_CHECK(cudaMalloc(&h->table_dev, sizeof(unsigned long long) * 66));
  CREATE_CHECK(cudaMalloc(&h->vol_dev, sizeof(VolumeArgs)));
  CREATE_CHECK(cudaMalloc(&h->rc_dev, sizeof(unsigned long long) * 10));
  CREATE_CHECK(cudaMallocHost(&h->host_pinned, 4096));
  if (p->eta_moves) {
    CREATE_CHECK(cudaMalloc(&h->eta, (size_t)(h->N / 4)));
    CREATE_CHECK(cudaMalloc(&h->eta_table_dev, sizeof(unsigned long long) * 18));
  }

  uint64_t table[66];
  threshold_table3(p, table);
  h->cmp64 = false;
  for (int i = 0; i < 66; ++i)
    if (table[i] == 0) h->cmp64 = true;
  VolumeArgs va;
  fill_volume_args3(p, h->N, d2, mult, &va);
  CREATE_CHECK(cudaMemcpyAsync(h->table_dev, table, sizeof(table), cudaMemcpyHostToDevice,
                               h->stream));
  CREATE_CHECK(cudaMemcpyAsync(h->vol_dev, &va, sizeof(va), cudaMemcpyHostToDevice, h->stream));
  CREATE_CHECK(cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));

  Args3& A = h->args;
  A.state = h->state;
  A.ctrl = h->ctrl;
  A.table = h->table_dev;
  A.vol = h->vol_dev;
  A.ring = h->ring;
  A.ring_cap = h->ring_cap;
  A.keys = make_round_keys(p->seed);
  A.L = L;
  A.L2 = L * L;
  A.N = (uint32_t)h->N;
  A.groups = (uint32_t)((h->N + 3) / 4);
  A.G = L / 4u;
  A.q = (uint32_t)p->q;
  h->aligned = (L % 4u) == 0u;
  A.div_G = make_fastdiv(h->aligned ? A.G : 1u);
  A.div_L = make_fastdiv(L);
  A.div_L2 = make_fastdiv(L * L);
  A.eta = h->eta;
  A.eta_table = h->eta_table_dev;
  cube_matchings(A.masks);
  A.H = L / 2u;
  A.ncube = p->eta_moves ? (uint32_t)(h->N / 4) : 0u;
  A.div_H = make_fastdiv(A.H > 0u ? A.H : 1u);
  if (p->eta_moves) {
    unsigned long long et[18];
    eta_table3(p, et);
    CREATE_CHECK(cudaMemcpyAsync(h->eta_table_dev, et, sizeof(et), cudaMemcpyHostToDevice,
                                 h->stream));
  }

  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pass_kernel(h->aligned, h->cmp64),
                                                    kThreads3, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const long long blocks = ((long long)A.groups + kThreads3 - 1) / kThreads3;
  h->grid = (int)std::max<long long>(1, std::min<long long>(blocks, (long long)sm_count() * per_sm));
  h->resident = resident3_auto(A, h->cmp64);
  h->grid_count = (int)std::max<long long>(
      1, std::min<long long>((h->N + kThreads3 - 1) / kThreads3, (long long)sm_count() * 8));
  h->grid_eta = (int)std::max<long long>(
      1, std::min<long long>((h->N / 4 + kThreads3 - 1) / kThreads3, (long long)sm_count() * 8));

  const int gi = (int)std::max<long long>(
      1, std::min<long long>(((long long)A.groups + kThreads3 - 1) / kThreads3,
                             (long long)sm_count() * 8));
  k_init3<<<gi, kThreads3, 0, h->stream>>>(h->state, A.N, A.groups, A.q,
                                            p->init == CVF_INIT_RANDOM ? 1 : 0, A.keys);
  if (p->eta_moves)
    k_eta_init3<<<h->grid_eta, kThreads3, 0, h->stream>>>(h->eta, A.ncube,
                                                           p->init == CVF_INIT_RANDOM ? 1 : 0,
                                                           A.keys);
  k_set_ctrl<<<1, 32, 0, h->stream>>>(h->vol_dev, h->ctrl, (double)h->N * p->v_iso_init, 0,
                                      h->N);
  rc = recount_into_ctrl3(h);
  if (rc) {
    release3(h);
    return rc;
  }
  CREATE_CHECK(cudaGetLastError());
  CREATE_CHECK(cudaStreamSynchronize(h->stream));
#undef CREATE_CHECK
  *out = h;
  return CVF_OK;
}

int cvf3_sweep(cvf3_handle* h, int64_t n_sweeps, int32_t record_every) {
  NvtxRange nvtx_range("cvf3_sweep");
  if (!h) return set_error(CVF_EINVAL, "handle is NULL");
  if (n_sweeps < 0 || record_every < 0)
    return set_error(CVF_EINVAL, "n_sweeps=%lld, record_every=%d must be >= 0",
                     (long long)n_sweeps, record_every);
  if (n_sweeps == 0) return CVF_OK;
  k_set_record<<<1, 32, 0, h->stream>>>(h->ctrl, record_every);
  if (h->resident) {
    constexpr long long kChunk = 1 << 16;
    if (!h->res_ctas) h->res_ctas = resident3_ctas(h->args, h->cmp64);
    for (long long done = 0; done < n_sweeps; done += kChunk)
      CVF_CUDA_CHECK(launch_resident3(h->args, h->cmp64, h->res_ctas,
                                      std::min(kChunk, n_sweeps - done), h->stream));
    return CVF_OK;
  }
  long long left = n_sweeps;
  if (left >= kGraphSteps3) {
    const int rc = build_graph3(h);
    if (rc) return rc;
    while (left >= kGraphSteps3) {
      CVF_CUDA_CHECK(cudaGraphLaunch(h->graph, h->stream));
      left -= kGraphSteps3;
    }
  }
  for (; left > 0; --left) enqueue_step3(h, h->stream);
  CVF_CUDA_CHECK(cudaGetLastError());
  return CVF_OK;
}

int cvf3_observables(cvf3_handle* h, cvf_obs* out) {
  NvtxRange nvtx_range("cvf3_observables");
  if (!h || !out) return set_error(CVF_EINVAL, "NULL argument");
  CVF_CUDA_CHECK(cudaMemsetAsync(h->rc_dev, 0, sizeof(unsigned long long) * 10, h->stream));
  k_count3<<<h->grid_count, kThreads3, 0, h->stream>>>(h->state, h->args.L, h->args.L2,
                                                        h->args.N, h->args.div_L, h->args.div_L2,
                                                        nullptr, h->rc_dev);
  k_observables3<<<1, 32, 0, h->stream>>>(h->vol_dev, h->ctrl, h->rc_dev, h->obs_dev);
  CVF_CUDA_CHECK(cudaGetLastError());
  CVF_CUDA_CHECK(cudaMemcpyAsync(h->host_pinned, h->obs_dev, sizeof(cvf_obs),
                                 cudaMemcpyDeviceToHost, h->stream));
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  std::memcpy(out, h->host_pinned, sizeof(cvf_obs));
  return status_error(out->status);
}

int cvf3_drain_series(cvf3_handle* h, cvf_obs* host, int64_t cap, int64_t* n) {
  NvtxRange nvtx_range("cvf3_drain_series");
  if (!h || !n || cap < 0 || (cap > 0 && !host)) return set_error(CVF_EINVAL, "bad argument");
  *n = 0;
  Ctrl c;
  CVF_CUDA_CHECK(cudaMemcpyAsync(h->host_pinned, h->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost,
                                 h->stream));
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  std::memcpy(&c, h->host_pinned, sizeof(Ctrl));
  int status = CVF_OK;
  if (c.ring_head - h->ring_tail > h->ring_cap) {
    h->ring_tail = c.ring_head - h->ring_cap;
    status = set_error(CVF_EOVERFLOW, "observable ring overwrote unread records");
  }
  const long long take = std::min<long long>(c.ring_head - h->ring_tail, cap);
  long long done = 0;
  while (done < take) {
    const long long slot = (h->ring_tail + done) % h->ring_cap;
    const long long chunk = std::min<long long>(take - done, h->ring_cap - slot);
    CVF_CUDA_CHECK(cudaMemcpyAsync(host + done, h->ring + slot, sizeof(cvf_obs) * chunk,
                                   cudaMemcpyDeviceToHost, h->stream));
    done += chunk;
  }
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  h->ring_tail += take;
  *n = take;
  return status;
}

int cvf3_get_state(cvf3_handle* h, uint32_t* host, size_t n) {
  NvtxRange nvtx_range("cvf3_get_state");
  if (!h || !host) return set_error(CVF_EINVAL, "NULL argument");
  if ((long long)n != h->N) return set_error(CVF_EINVAL, "n=%zu, lattice has %lld cells", n, h->N);
  CVF_CUDA_CHECK(cudaMemcpyAsync(host, h->state, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost,
                                 h->stream));
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  for (size_t i = 0; i < n; ++i) host[i] &= kArmBits;  // drop the eta copies
  return CVF_OK;
}

int cvf3_get_window(cvf3_handle* h, int32_t x0, int32_t y0, int32_t z0, int32_t W, int32_t H,
                    int32_t D, uint32_t* host) {
  NvtxRange nvtx_range("cvf3_get_window");
  if (!h || !host) return set_error(CVF_EINVAL, "NULL argument");
  const long long L = h->p.L;
  if (W < 1 || H < 1 || D < 1 || x0 < 0 || y0 < 0 || z0 < 0 || (long long)x0 + W > L ||
      (long long)y0 + H > L || (long long)z0 + D > L)
    return set_error(CVF_EINVAL, "box (%d, %d, %d) + (%d, %d, %d) outside the %lld^3 cube", x0,
                     y0, z0, W, H, D, L);
  const size_t row = sizeof(uint32_t) * (size_t)L;
  for (int32_t z = 0; z < D; ++z) {
    const uint32_t* src = h->state + ((size_t)(z0 + z) * (size_t)L + (size_t)y0) * (size_t)L +
                          (size_t)x0;
    CVF_CUDA_CHECK(cudaMemcpy2DAsync(host + (size_t)z * H * W, sizeof(uint32_t) * (size_t)W, src,
                                     row, sizeof(uint32_t) * (size_t)W, (size_t)H,
                                     cudaMemcpyDeviceToHost, h->stream));
  }
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  const size_t n = (size_t)W * H * D;
  for (size_t i = 0; i < n; ++i) host[i] &= kArmBits;  // drop the eta copies
  return CVF_OK;
}

int cvf3_set_state(cvf3_handle* h, const uint32_t* host, size_t n, double V_iso, int64_t sweep) {
  NvtxRange nvtx_range("cvf3_set_state");
  if (!h || !host) return set_error(CVF_EINVAL, "NULL argument");
  if ((long long)n != h->N) return set_error(CVF_EINVAL, "n=%zu, lattice has %lld cells", n, h->N);
  if (!(V_iso >= (double)h->N) || !std::isfinite(V_iso))
    return set_error(CVF_EINVAL, "V_iso=%g must be >= N=%lld (hard core)", V_iso, h->N);
  if (sweep < 0) return set_error(CVF_EINVAL, "sweep=%lld must be >= 0", (long long)sweep);
  const uint32_t q = (uint32_t)h->p.q;
  // two cells per 64-bit load: bits outside the arms' sigma bits must be
  // clear, and then a nibble v is >= q exactly when v + 8 - q sets its bit 3
  const uint64_t keep = ((uint64_t)kArmBits << 32) | kArmBits;
  const uint64_t G = ((uint64_t)0x888888u << 32) | 0x888888u;
  const uint64_t add = (uint64_t)(8u - q) * (((uint64_t)0x111111u << 32) | 0x111111u);
  size_t i = 0;
  for (; i + 2 <= n; i += 2) {
    uint64_t x;
    std::memcpy(&x, host + i, sizeof(x));
    if ((x & ~keep) | ((x + add) & G)) break;
  }
  for (; i < n; ++i) {
    const uint32_t w = host[i];
    bool ok = (w & ~kArmBits) == 0u;
    for (int a = 0; a < 6 && ok; ++a) ok = ((w >> (4 * a)) & 7u) < q;
    if (!ok)
      return set_error(CVF_EINVAL, "word %zu = 0x%x: arms must be < q=%u, bits 4a+3 and 24..31 zero",
                       i, w, q);
  }
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  CVF_CUDA_CHECK(cudaMemcpyAsync(h->state, host, sizeof(uint32_t) * n, cudaMemcpyHostToDevice,
                                 h->stream));
  k_set_ctrl<<<1, 32, 0, h->stream>>>(h->vol_dev, h->ctrl, V_iso, sweep, h->N);
  int rc = recount_into_ctrl3(h);
  if (rc) return rc;
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  h->ring_tail = 0;
  return CVF_OK;
}

int cvf3_get_eta(cvf3_handle* h, uint8_t* host, size_t n) {
  NvtxRange nvtx_range("cvf3_get_eta");
  if (!h || !host) return set_error(CVF_EINVAL, "NULL argument");
  if (!h->eta) return set_error(CVF_EINVAL, "the lattice was created without eta moves");
  if ((long long)n != h->N / 4)
    return set_error(CVF_EINVAL, "n=%zu, the lattice has %lld cubes", n, h->N / 4);
  CVF_CUDA_CHECK(cudaMemcpyAsync(host, h->eta, n, cudaMemcpyDeviceToHost, h->stream));
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  return CVF_OK;
}

int cvf3_set_eta(cvf3_handle* h, const uint8_t* host, size_t n) {
  NvtxRange nvtx_range("cvf3_set_eta");
  if (!h || !host) return set_error(CVF_EINVAL, "NULL argument");
  if (!h->eta) return set_error(CVF_EINVAL, "the lattice was created without eta moves");
  if ((long long)n != h->N / 4)
    return set_error(CVF_EINVAL, "n=%zu, the lattice has %lld cubes", n, h->N / 4);
  for (size_t i = 0; i < n; ++i)
    if (host[i] > 8u)
      return set_error(CVF_EINVAL, "cube %zu: configuration %u, need 0..8", i, (unsigned)host[i]);
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  CVF_CUDA_CHECK(cudaMemcpyAsync(h->eta, host, n, cudaMemcpyHostToDevice, h->stream));
  int rc = recount_into_ctrl3(h);
  if (rc) return rc;
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  return CVF_OK;
}

int cvf3_recount(cvf3_handle* h, int64_t* n_hb_raw, int64_t* n_sigma) {
  NvtxRange nvtx_range("cvf3_recount");
  if (!h || !n_hb_raw || !n_sigma) return set_error(CVF_EINVAL, "NULL argument");
  CVF_CUDA_CHECK(cudaMemsetAsync(h->rc_dev, 0, sizeof(unsigned long long) * 10, h->stream));
  k_count3<<<h->grid_count, kThreads3, 0, h->stream>>>(h->state, h->args.L, h->args.L2,
                                                        h->args.N, h->args.div_L, h->args.div_L2,
                                                        h->rc_dev + 8, nullptr);
  CVF_CUDA_CHECK(cudaGetLastError());
  unsigned long long r[2];
  CVF_CUDA_CHECK(cudaMemcpyAsync(h->host_pinned, h->rc_dev + 8, sizeof(r), cudaMemcpyDeviceToHost,
                                 h->stream));
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  std::memcpy(r, h->host_pinned, sizeof(r));
  *n_hb_raw = (int64_t)r[0];
  *n_sigma = (int64_t)r[1];
  return CVF_OK;
}

int cvf3_set_resident(cvf3_handle* h, int32_t mode) {
  if (!h) return set_error(CVF_EINVAL, "handle is NULL");
  if (mode < -1 || mode > 1) return set_error(CVF_EINVAL, "mode %d: need -1, 0 or 1", mode);
  const bool fits = resident3_fits(h->args, h->cmp64);
  if (mode == 1 && !fits)
    return set_error(CVF_EINVAL, "the resident form needs L a multiple of %d, %d <= L <= %d",
                     kRes3Ctas, 2 * kRes3Ctas, kRes3MaxSide);
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  h->resident = (mode == 1) || (mode == -1 && resident3_auto(h->args, h->cmp64));
  return CVF_OK;
}

int cvf3_get_resident(cvf3_handle* h, int32_t* resident) {
  if (!h || !resident) return set_error(CVF_EINVAL, "NULL argument");
  *resident = h->resident ? 1 : 0;
  return CVF_OK;
}

int cvf3_state_device_ptr(cvf3_handle* h, void** dev_ptr) {
  if (!h || !dev_ptr) return set_error(CVF_EINVAL, "NULL argument");
  *dev_ptr = h->state;
  return CVF_OK;
}

int cvf3_destroy(cvf3_handle* h) {
  if (!h) return CVF_OK;
  cudaStreamSynchronize(h->stream);
  release3(h);
  return CVF_OK;
}

}  // extern "C"
