// cvf_lattice.cu -- single-lattice path of the CVF library: kernels for the
// initial configuration, the checkerboard and layered Metropolis sweeps
// (Sec. II.C), the N_HB / N_sigma reductions (Eq. H), the FP64 volume move
// (Sec. II.B) and the observables, plus the C-ABI entry points that drive
// them with CUDA graphs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "cvf.h"
#include "cvf_device.cuh"
#include "cvf_host.h"
#include "cvf_lattice.cuh"
#include "cvf_tile.cuh"
#include "cvf_tma.cuh"
#include <cudaTypedefs.h>

using namespace cvf;

namespace cvf {

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------

// Initial configuration: sigma_a(c) = floor(w_a q / 2^32) with w =
// Philox((c, 0, 0, tag 2)), or every sigma = 0 (ordered, all bonds formed).
__global__ void k_init(uint16_t* __restrict__ state, int32_t L, uint32_t q, int random,
                       RoundKeys K) {
  const long long N = (long long)L * L;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    uint32_t w = 0;
    if (random) {
      const Words4 r = philox((uint32_t)c, 0u, 0u, kTagInit, K);
      w = __umulhi(r.x, q) | (__umulhi(r.y, q) << 4) | (__umulhi(r.z, q) << 8) |
          (__umulhi(r.w, q) << 12);
    }
    state[c] = (uint16_t)w;
  }
}

// Full recount of N_HB_raw (the +x and +y bond of every cell) and N_sigma
// (equal pairs inside every cell); adds the totals to out[0], out[1].  With
// ctl != nullptr the lattice read is the half of the state pair that the
// running step writes (buffer (sweep + 1) & 1).
__global__ void __launch_bounds__(kThreads) k_recount(const uint16_t* __restrict__ base,
                                                      int32_t L, const Ctrl* ctl,
                                                      unsigned long long* out) {
  const long long N = (long long)L * L;
  const uint16_t* state = base;
  if (ctl) state = base + (size_t)((ctl->sweep + 1) & 1) * N;
  uint32_t hb = 0, pairs = 0, unused = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(c / L), x = (int)(c - (long long)y * L);
    const uint32_t w = state[c];
    const uint32_t wxp = state[(long long)y * L + (x + 1 == L ? 0 : x + 1)];
    const uint32_t wyp = state[(long long)(y + 1 == L ? 0 : y + 1) * L + x];
    hb += (uint32_t)(arm_of(w, 0) == arm_of(wxp, 1)) + (uint32_t)(arm_of(w, 2) == arm_of(wyp, 3));
    pairs += cell_pairs(w);
  }
  block_sum3<kThreads>(hb, pairs, unused);
  if (threadIdx.x == 0) {
    atomicAdd(&out[0], (unsigned long long)hb);
    atomicAdd(&out[1], (unsigned long long)pairs);
  }
}

// Adopt recounted totals as the committed counts; clear the accumulators.
__global__ void k_commit_counts(Ctrl* ctl) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl->n_hb_raw = (long long)ctl->acc_hb;
    ctl->n_coop = (long long)ctl->acc_pairs;
    ctl->acc_hb = 0;
    ctl->acc_pairs = 0;
    ctl->acc_moves = 0;
    ctl->done = 0;
  }
}

__global__ void k_set_ctrl(const VolumeArgs* __restrict__ V, Ctrl* ctl, double V_iso,
                           long long sweep, long long N) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl->sweep = sweep;
    ctl->V_iso = V_iso;
    ctl->u_cell = lj_cell_energy(*V, V_iso / (double)N);
    ctl->g = (V_iso / (double)N < 2.0) ? 1 : 0;
    ctl->ahead_state = 0;
    ctl->tile_next = 0;
    ctl->acc_sigma = 0;
    ctl->acc_volume = 0;
    ctl->acc_hb = 0;
    ctl->acc_pairs = 0;
    ctl->acc_moves = 0;
    ctl->done = 0;
    ctl->ring_head = 0;
    ctl->record_every = 0;
  }
}

__global__ void k_set_record(Ctrl* ctl, int record_every) {
  if (threadIdx.x == 0 && blockIdx.x == 0) ctl->record_every = record_every;
}

// The volume move of the next step from the committed state (run once after
// the lattice or the counters are (re)set; afterwards every step's end
// prepares the move of the following step).
__global__ void k_volume_prologue(const VolumeArgs* __restrict__ V, Ctrl* ctl, RoundKeys K) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    VolumeResult r;
    volume_decide(*V, ctl->sweep, ctl->V_iso, ctl->u_cell, ctl->g, ctl->n_hb_raw, K, &r);
    ctl->next_V = r.V;
    ctl->next_u = r.u;
    ctl->next_g = r.g;
    ctl->next_acc = r.accepted;
    ctl->ahead_state = 0;
  }
}

__global__ void k_observables(const VolumeArgs* __restrict__ V, const Ctrl* ctl,
                              const unsigned long long* hist, cvf_obs* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    Ctrl c = *ctl;
    if (hist) c.n_coop = (long long)hist[8];  // counted now from the lattice
    cvf_obs o = make_obs(*V, &c);
    if (hist)
      for (int v = 0; v < 8; ++v) o.n_state[v] = (long long)hist[v];
    *out = o;
  }
}

// The first word of w[0, n) that is not a valid cell for q (a spare bit set or
// an arm >= q), as an atomic minimum into *first (left at its initial value,
// the caller's all-ones, when every word is valid).
__global__ void __launch_bounds__(kThreads) k_first_invalid(const uint16_t* __restrict__ w,
                                                            long long n, uint32_t q,
                                                            unsigned long long* first) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const uint32_t x = w[i];
    if ((x & 0x8888u) || (x & 7u) >= q || ((x >> 4) & 7u) >= q || ((x >> 8) & 7u) >= q ||
        ((x >> 12) & 7u) >= q)
      atomicMin(first, (unsigned long long)i);
  }
}

// N_q' of a lattice (the number of sigma variables in each state) added to
// out[0..8), and its equal in-cell pairs (N_sigma) added to out[8].
__global__ void __launch_bounds__(kThreads) k_histogram(const uint16_t* __restrict__ state,
                                                        long long N, unsigned long long* out) {
  __shared__ unsigned long long s_cnt[9];
  if (threadIdx.x < 9) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  uint32_t c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  uint32_t pairs = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const uint32_t w = state[i];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const uint32_t v = (w >> (4 * a)) & 7u;
#pragma unroll
      for (int k = 0; k < 8; ++k) c[k] += (v == (uint32_t)k) ? 1u : 0u;
    }
    pairs += cell_pairs(w);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k)
    if (c[k]) atomicAdd(&s_cnt[k], (unsigned long long)c[k]);
  if (pairs) atomicAdd(&s_cnt[8], (unsigned long long)pairs);
  __syncthreads();
  if (threadIdx.x < 9 && s_cnt[threadIdx.x]) atomicAdd(&out[threadIdx.x], s_cnt[threadIdx.x]);
}

// ---------------------------------------------------------------------------
// Checkerboard sweep, both colours in one launch (the tile algorithm is in
// cvf_tile.cuh).  Blocks take tiles from a per-step atomic counter; block 0
// instead decides the next step's volume move early (it depends on the bonds
// only when the gate would change).  Per thread the accepted moves of the
// tile cells and their changes of N_HB_raw and N_sigma are summed,
// block-reduced and added with one atomic each; the last block adds the
// changes to the committed counts and closes the step.
// ---------------------------------------------------------------------------
// Bounded wait for a TMA stage (the copies complete in microseconds; the
// limit only guards against a copy that never lands).
constexpr uint32_t kTmaWaitLimit = 1u << 26;

// Tile shapes of the single-lattice sweep (rows x 32-bit words): the large
// tile for large lattices, smaller ones so that mid-size lattices still
// give every resident block tiles to take.
template <int TILE>
struct TileShape {
  static constexpr int R = (TILE == 0) ? 64 : (TILE == 1) ? 32 : 16;
  static constexpr int W = (TILE == 0) ? 64 : 32;
};
constexpr int kNumSweepTiles = 3;
// colour loops: one row loop per half and per recorded / unrecorded step,
// two cells per iteration in colour 1 only (at 4096^2: 522 sigma-updates/ns;
// 520 with one cell per iteration in both colours, 500-503 with two cells per
// iteration and the half a runtime value, 458 with one loop per half and two
// cells per iteration in colour 0)
constexpr int kSweepShape = kHalfRows | kUnroll1 | kSplitRec;

// WALK: every tile of the lattice is full and the rows are 16-byte aligned
// (L a multiple of the tile height and of 2 x the tile width, Lh of 4), so
// the colour phases take the column-walking form (colour0_walk /
// colour1_walk); a separate instantiation, since one kernel holding both forms
// spills.
template <int RNG_WORDS, bool CMP64, int TILE, bool WALK>
__global__ void __launch_bounds__(kThreads, kSweepBlocksPerSM)
    k_sweep_tiled(const __grid_constant__ LatticeArgs A, const __grid_constant__ CUtensorMap tm0,
                  const __grid_constant__ CUtensorMap tm1) {
  constexpr int kTileRows = TileShape<TILE>::R, kTileWords = TileShape<TILE>::W;
  // the volume block uses the tile buffers for its copy of the parameters
  __shared__ union {
    TileSmem<kTileRows, kTileWords> tile;
    VolumeArgs vol;
  } U;
  TileSmem<kTileRows, kTileWords>& S = U.tile;
  __shared__ Tables2 Tb;
  __shared__ int s_tile, s_next;
  __shared__ uint32_t s_hist4[4];
  __shared__ alignas(8) uint64_t s_bar;
  pdl_wait();     // the previous step's launch has completed (programmatic launch)
  pdl_trigger();  // the next step's launch may start while this one runs
  Ctrl* ctl = A.ctrl;
  const int g = ctl->next_g;
  const long long step = ctl->sweep;
  if (blockIdx.x == 0) {
    // the volume block: decide the next step's volume move now when it does
    // not depend on this step's bonds, while the other blocks sweep (the
    // parameters staged into the unused tile buffers first)
    VolumeArgs* sV = &U.vol;
    __shared__ double s_xch;
    stage_volume_args(sV, A.vol);
    __syncthreads();
    if (threadIdx.x < 64) {  // warps 0 and 1: the move on two FP64 pipes
      VolumeResult r;
      const bool ok = volume_decide_pair<3>((int)(threadIdx.x >> 5), *sV, step + 1, ctl->next_V,
                                            ctl->next_u, ctl->next_g, -1, A.keys, &r, &s_xch);
      if (threadIdx.x == 0 && ok) {
        ctl->ahead_V = r.V;
        ctl->ahead_u = r.u;
        ctl->ahead_g = r.g;
        ctl->ahead_acc = r.accepted;
        ctl->ahead_state = 1;
      }
    }
    if (last_block(&ctl->done) && threadIdx.x == 0)
      finalize_step<true>(*A.vol, ctl, A.ring, A.ring_cap, A.keys);
    return;
  }
  fill_rows2(Tb, A.table24, g);
  fill_prop2(Tb, A.q);
  const long long N = (long long)A.L * A.L;
  StepView<KeysRound> v;
  v.src = reinterpret_cast<const uint32_t*>(A.state + (size_t)(step & 1) * N);
  v.dst = reinterpret_cast<uint32_t*>(A.state + (size_t)((step + 1) & 1) * N);
  v.L = A.L;
  v.Lh = A.L >> 1;
  v.q = A.q;
  v.s_lo = (uint32_t)((unsigned long long)step & 0xFFFFFFFFu);
  v.s_hi = (uint32_t)((unsigned long long)step >> 32);
  v.keys.K = &A.keys;
  v.err = &ctl->error;
  const CUtensorMap* tmap = (step & 1) ? &tm1 : &tm0;  // map of the source buffer
  const int tiles_x = (v.Lh + kTileWords - 1) / kTileWords;
  const int ntiles = tiles_x * ((v.L + kTileRows - 1) / kTileRows);
  const bool rec = step_recorded(ctl->record_every, step);
  TileCounts cnt{0, 0, 0};
  if (threadIdx.x < 4) s_hist4[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    // the first tile of tile block b is b - 1 (no round trip to the counter);
    // the counter hands out the tiles after the first gridDim.x - 1
    s_tile = (int)blockIdx.x - 1;
  }
  __syncthreads();

  // Start the copy of tile t into S.in: one TMA box for tiles whose halo lies
  // inside the lattice, 4-byte cp.async copies otherwise (periodic wrap).
  // Returns whether the copy goes through the barrier.
  auto stage = [&](int t) -> bool {
    const TileGeom gm = tile_geom<kTileRows, kTileWords>(v.L, v.Lh, (t / tiles_x) * kTileRows,
                                                         (t % tiles_x) * kTileWords);
    const bool tma = A.use_tma && gm.th == kTileRows && gm.tw == kTileWords && gm.p0 >= 4 &&
                     gm.p0 + kTileWords + 4 <= v.Lh && gm.y0 >= 2 &&
                     gm.y0 + kTileRows + 2 <= v.L;
    if (tma) {
      if (threadIdx.x == 0) {
        fence_proxy_async_shared();
        // the box's x (words) must be a multiple of 4 (16 bytes) and the box
        // inside the lattice; a debug build that finds otherwise arrives
        // without a copy, so the wait still ends
        if (dcheck(((gm.p0 - 4) & 3) == 0 && gm.p0 - 4 >= 0 && gm.y0 - 2 >= 0 &&
                       gm.p0 - 4 + kTileWords + 8 <= v.Lh && gm.y0 - 2 + kTileRows + 4 <= v.L,
                   v.err, kSiteTma)) {
          mbar_arrive_expect_tx(&s_bar, (uint32_t)sizeof(S.in));
          tma_load_2d(&S.in[0][0], tmap, gm.p0 - 4, gm.y0 - 2, &s_bar);
        } else {
          mbar_arrive_expect_tx(&s_bar, 0u);
        }
      }
    } else {
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
      for (int rr = warp; rr < gm.th + 4; rr += kThreads / 32) {
        int y = gm.y0 + rr - 2;
        y = (y < 0) ? y + v.L : (y >= v.L ? y - v.L : y);
        const uint32_t* row = v.src + (size_t)y * v.Lh;
        for (int jj = lane; jj < gm.tw + 2; jj += 32) {
          int p = gm.p0 + jj - 1;
          p = (p < 0) ? p + v.Lh : (p >= v.Lh ? p - v.Lh : p);
          if (dcheck(y >= 0 && y < v.L && p >= 0 && p < v.Lh && rr < kTileRows + 4 &&
                         jj + kInColOff < kTileWords + 8,
                     v.err, kSiteStage))
            cp_async4(&S.in[rr][jj + kInColOff], row + p);
        }
      }
      cp_async_commit();
    }
    return tma;
  };

  uint32_t parity = 0;
  int t = s_tile;
  bool t_tma = (t < ntiles) ? stage(t) : false;
  while (t < ntiles) {
    // wait for tile t's input
    if (t_tma) {
      uint32_t spins = 0;
      while (!mbar_try_wait(&s_bar, parity)) {
        if (++spins > kTmaWaitLimit) {
          atomicOr(&ctl->error, 1u);
          break;
        }
      }
      parity ^= 1u;
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    const TileGeom gm = tile_geom<kTileRows, kTileWords>(v.L, v.Lh, (t / tiles_x) * kTileRows,
                                                         (t % tiles_x) * kTileWords);
    if constexpr (WALK) {
      if (rec)
        colour0_walk<RNG_WORDS, CMP64, kTileRows, kTileWords, kThreads, true, 1>(v, gm, S, Tb, cnt,
                                                                               s_hist4);
      else
        colour0_walk<RNG_WORDS, CMP64, kTileRows, kTileWords, kThreads, false, 1>(v, gm, S, Tb, cnt,
                                                                                nullptr);
    } else {
      colour0<RNG_WORDS, CMP64, kTileRows, kTileWords, kThreads, kSweepShape>(
          v, gm, S, Tb, cnt, rec ? s_hist4 : nullptr);
    }
    if (threadIdx.x == 0) s_next = (int)(atomicAdd(&ctl->tile_next, 1u) + gridDim.x - 1u);
    __syncthreads();  // S.in is free: fetch the next tile while colour 1 runs
    const int t2 = s_next;
    const bool t2_tma = (t2 < ntiles) ? stage(t2) : false;
    if constexpr (WALK) {
      if (rec)
        colour1_walk<RNG_WORDS, CMP64, kTileRows, kTileWords, kThreads, true, 1>(v, gm, S, Tb, cnt,
                                                                               s_hist4);
      else
        colour1_walk<RNG_WORDS, CMP64, kTileRows, kTileWords, kThreads, false, 1>(v, gm, S, Tb, cnt,
                                                                                nullptr);
    } else {
      colour1<RNG_WORDS, CMP64, kTileRows, kTileWords, kThreads, kSweepShape>(
          v, gm, S, Tb, cnt, rec ? s_hist4 : nullptr);
    }
    if (rec) {
      __syncthreads();
      hist_flush(s_hist4, ctl->acc_hist);
    }
    __syncthreads();  // S.mid is free for the next tile
    t = t2;
    t_tma = t2_tma;
  }
  uint32_t dhb = (uint32_t)cnt.dhb(), dc = (uint32_t)cnt.dc(), nacc = cnt.nacc;
  block_sum3<kThreads>(dhb, dc, nacc);  // two's complement sums
  if (threadIdx.x == 0) {
    atomicAdd(&ctl->acc_hb, (unsigned long long)(long long)(int)dhb);
    atomicAdd(&ctl->acc_pairs, (unsigned long long)(long long)(int)dc);
    atomicAdd(&ctl->acc_moves, (unsigned long long)nacc);
  }
  if (last_block(&ctl->done) && threadIdx.x == 0)
    finalize_step<true>(*A.vol, ctl, A.ring, A.ring_cap, A.keys);
}

// ---------------------------------------------------------------------------
// Layered schedule (the paper's own scheme, Sec. II.C): the four arm domains
// one after the other, in a Fisher-Yates order drawn from Philox((2^32-2,
// step, tag 4)).  A pass over arm a reads, besides the cell, only arm a^1 of
// its neighbour in direction a, which only the pass over a^1 changes; so
// consecutive passes without an opposite pair share a launch, each thread
// taking its two cells (one word) through them in registers (every partner
// arm it reads is constant during the launch).  The order is cut before the
// first arm whose opposite is already in the launch: 2 or 3 launches; every
// step enqueues kLayerLaunches, the unused ones return at once, the last one
// commits the step.  Launch 0 reads the step's source buffer and writes every
// word of the other buffer; the later launches update that buffer in place.
// A cell's draws are its Philox((c, step, 0)) words (and tag 1 with two
// words per update), recomputed in every launch that updates the cell.
// ---------------------------------------------------------------------------
constexpr int kLayerLaunches = 3;

// Plan word: bits 2i..2i+1 the arm of pass i, bit 8 + i set when pass i
// opens a new launch (i = 1..3).
__device__ uint32_t layer_plan(long long step, const RoundKeys& K) {
  const Words4 r = philox(kCellLayers, (uint32_t)((unsigned long long)step & 0xFFFFFFFFu),
                          (uint32_t)((unsigned long long)step >> 32), kTagLayers, K);
  const uint32_t rw[4] = {r.x, r.y, r.z, r.w};
  int order[4] = {0, 1, 2, 3};
  for (int i = 3; i >= 1; --i) {
    const int j = (int)__umulhi(rw[3 - i], (uint32_t)(i + 1));
    const int t = order[i];
    order[i] = order[j];
    order[j] = t;
  }
  uint32_t plan = 0, in_launch = 0;
  for (int i = 0; i < 4; ++i) {
    const int a = order[i];
    if (in_launch & (1u << (a ^ 1))) {
      plan |= 1u << (8 + i);
      in_launch = 0;
    }
    in_launch |= 1u << a;
    plan |= (uint32_t)a << (2 * i);
  }
  return plan;
}

__device__ int layer_plan_arms(uint32_t plan, int j, int* arms) {
  int launch = 0, n = 0;
  for (int i = 0; i < 4; ++i) {
    if (i > 0 && ((plan >> (8 + i)) & 1u)) ++launch;
    if (launch == j && n < 2) arms[n++] = (int)((plan >> (2 * i)) & 3u);
  }
  return n;
}

// The partner of arm a of the cell in half `hi` of word `own` (at column p
// of row y), moved to bits 16..18: arm a^1 of the neighbour in direction a.
__device__ __forceinline__ uint32_t layer_partner(int a, int hi, uint32_t own, const uint32_t* buf,
                                                  uint32_t y, uint32_t p, uint32_t L,
                                                  uint32_t Lh) {
  if (a == 0) {  // +x: arm 1 of the cell to the right
    if (!hi) return (own >> 4) & 0x70000u;
    const uint32_t pn = (p + 1u == Lh) ? 0u : p + 1u;
    return (buf[y * Lh + pn] << 12) & 0x70000u;
  }
  if (a == 1) {  // -x: arm 0 of the cell to the left
    if (hi) return (own << 16) & 0x70000u;
    const uint32_t pm = (p == 0u) ? Lh - 1u : p - 1u;
    return buf[y * Lh + pm] & 0x70000u;
  }
  if (a == 2) {  // +y: arm 3 of the cell below, same half
    const uint32_t yn = (y + 1u == L) ? 0u : y + 1u;
    const uint32_t wv = buf[yn * Lh + p];
    return hi ? (wv >> 12) & 0x70000u : (wv << 4) & 0x70000u;
  }
  const uint32_t ym = (y == 0u) ? L - 1u : y - 1u;  // -y: arm 2 of the cell above
  const uint32_t wv = buf[ym * Lh + p];
  return hi ? (wv >> 8) & 0x70000u : (wv << 8) & 0x70000u;
}

template <int RNG_WORDS, bool CMP64>
__global__ void __launch_bounds__(kThreads) k_layer(LatticeArgs A, int launch) {
  __shared__ Tables2 Tb;
  __shared__ int s_arm[2];
  __shared__ int s_n, s_rec;
  __shared__ uint32_t s_hist[8];
  Ctrl* ctl = A.ctrl;
  const bool fin = (launch == kLayerLaunches - 1);
  if (threadIdx.x == 0) {
    uint32_t plan;
    if (launch == 0) {
      plan = layer_plan(ctl->sweep, A.keys);
      if (blockIdx.x == 0) ctl->plan = (int)plan;
    } else {
      plan = (uint32_t)ctl->plan;
    }
    int arms[2] = {0, 0};
    const int n = layer_plan_arms(plan, launch, arms);
    s_n = n;
    s_arm[0] = arms[0];
    s_arm[1] = arms[1];
    const int nlaunch = 1 + __popc(plan >> 9);
    s_rec = (n > 0 && launch == nlaunch - 1 && step_recorded(ctl->record_every, ctl->sweep)) ? 1 : 0;
  }
  __syncthreads();
  const int n_arms = s_n;
  if (launch == 0 && blockIdx.x == 0) {
    // the volume block: the next step's move, decided now unless it depends on the bonds
    __shared__ VolumeArgs sV;
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
    if (fin && blockIdx.x == 0 && threadIdx.x == 0)
      finalize_step<true>(*A.vol, ctl, A.ring, A.ring_cap, A.keys);
    return;
  }
  const long long step = ctl->sweep;
  const int g = ctl->next_g;
  const bool rec = s_rec != 0;
  fill_rows2(Tb, A.table24, g);
  fill_prop2(Tb, A.q);
  if (threadIdx.x < 8) s_hist[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t L = (uint32_t)A.L, Lh = L >> 1;
  const long long N = (long long)L * L;
  const uint32_t* src = reinterpret_cast<const uint32_t*>(A.state + (size_t)(step & 1) * N);
  uint32_t* dst = reinterpret_cast<uint32_t*>(A.state + (size_t)((step + 1) & 1) * N);
  const uint32_t* in = (launch == 0) ? src : dst;  // the launch's input words
  const uint32_t s_lo = (uint32_t)((unsigned long long)step & 0xFFFFFFFFu);
  const uint32_t s_hi = (uint32_t)((unsigned long long)step >> 32);
  const int a0 = s_arm[0], a1 = s_arm[1];
  const uint32_t first_block = (launch == 0) ? 1u : 0u;
  const uint32_t nwords = (uint32_t)(N >> 1);
  TileCounts cnt{0, 0, 0};
  for (uint32_t wi = (blockIdx.x - first_block) * kThreads + threadIdx.x; wi < nwords;
       wi += (gridDim.x - first_block) * kThreads) {
    const uint32_t y = wi / Lh, p = wi - y * Lh;
    if (!dcheck(y < L && p < Lh, &ctl->error, kSiteLayer)) continue;
    const uint32_t own = in[wi];
    uint32_t out = own;
    uint32_t pk = 0;
#pragma unroll
    for (int hi = 0; hi < 2; ++hi) {
      uint32_t w = hi ? (own >> 16) : (own & 0xFFFFu);
      const uint32_t c = y * L + 2u * p + (uint32_t)hi;
      uint32_t acc[4], kk[4];
      cell_draws<RNG_WORDS>(c, s_lo, s_hi, A.keys, A.q, acc, kk);
      for (int k = 0; k < n_arms; ++k) {
        const int a = k ? a1 : a0;
        const uint32_t pa = layer_partner(a, hi, own, in, y, p, L, Lh);
        // the draws of arm a, selected without indexing the arrays at run time
        const uint32_t ua = (a == 0) ? acc[0] : (a == 1) ? acc[1] : (a == 2) ? acc[2] : acc[3];
        const uint32_t ka = (a == 0) ? kk[0] : (a == 1) ? kk[1] : (a == 2) ? kk[2] : kk[3];
        w = update_arm2<CMP64>(w, partner_operand(pa), ua, ka, (uint32_t)a, Tb, pk);
      }
      out = hi ? ((out & 0xFFFFu) | (w << 16)) : ((out & 0xFFFF0000u) | w);
    }
    cnt.add(pk);
    dst[wi] = out;
    if (rec) {
      // N_q' of the step's final cells: 16-bit lanes (state v, state v + 4)
      // summed over the converged lanes of the warp, added by the lowest
      const uint32_t h = count_word4(out & 0xFFFFu) + count_word4(out >> 16);
      const unsigned mask = __activemask();
      const int leader = __ffs(mask) - 1;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const uint32_t lanes = __reduce_add_sync(mask, (h >> (4 * v)) & 0x000F000Fu);
        if ((int)(threadIdx.x & 31) == leader) {
          if (lanes & 0xFFFFu) atomicAdd(&s_hist[v], lanes & 0xFFFFu);
          if (lanes >> 16) atomicAdd(&s_hist[v + 4], lanes >> 16);
        }
      }
    }
  }
  uint32_t dhb = (uint32_t)cnt.dhb(), dc = (uint32_t)cnt.dc(), nacc = cnt.nacc;
  block_sum3<kThreads>(dhb, dc, nacc);  // two's complement sums
  if (threadIdx.x == 0) {
    atomicAdd(&ctl->acc_hb, (unsigned long long)(long long)(int)dhb);
    atomicAdd(&ctl->acc_pairs, (unsigned long long)(long long)(int)dc);
    atomicAdd(&ctl->acc_moves, (unsigned long long)nacc);
  }
  if (rec) {
    __syncthreads();
    if (threadIdx.x < 8 && s_hist[threadIdx.x])
      atomicAdd(&ctl->acc_hist[threadIdx.x], (unsigned long long)s_hist[threadIdx.x]);
  }
  if (fin && last_block(&ctl->done) && threadIdx.x == 0)
    finalize_step<true>(*A.vol, ctl, A.ring, A.ring_cap, A.keys);
}

}  // namespace cvf

namespace cvf {

// Device threshold rows [g][(dN_HB+1)*8 + dN_sigma+3] (slot dN_sigma+3 = 7
// unused); returns true when some threshold is 0 (64-bit compares needed).
bool fill_table24(const cvf_params* p, unsigned long long table24[48]) {
  uint64_t table[42];
  threshold_table(p, table);
  std::memset(table24, 0, sizeof(unsigned long long) * 48);
  bool cmp64 = false;
  for (int g = 0; g < 2; ++g)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 7; ++j) {
        const uint64_t t = table[(g * 3 + i) * 7 + j];
        table24[g * 24 + i * 8 + j] = t;
        if (t == 0) cmp64 = true;
      }
  return cmp64;
}

// FP64 parameters and the LJ shell prefix sums (accumulated in increasing
// |d|^2: S12 of m/|d|^12, S6 of m/|d|^6).
void fill_volume_args(const cvf_params* p, long long N, const std::vector<int64_t>& d2,
                      const std::vector<int64_t>& mult, VolumeArgs* va) {
  std::memset(va, 0, sizeof(*va));
  va->N = N;
  va->epsilon = p->epsilon;
  va->cutoff2 = p->cutoff * p->cutoff;
  va->J = p->J;
  va->J_sigma = p->J_sigma;
  va->v_HB = p->v_HB;
  va->kT = p->kT;
  va->P = p->P;
  va->dV_max = p->dv_max_frac * ((double)N * p->v_iso_init);
  va->volume_moves = p->volume_moves;
  va->nshell = (int)d2.size();
  va->S12[0] = 0.0;
  va->S6[0] = 0.0;
  for (size_t i = 0; i < d2.size(); ++i) {
    va->shell_d2[i] = (double)d2[i];
    const int64_t d6 = d2[i] * d2[i] * d2[i];
    va->S12[i + 1] = va->S12[i] + (double)mult[i] / ((double)d6 * (double)d6);
    va->S6[i + 1] = va->S6[i] + (double)mult[i] / (double)d6;
  }
}

}  // namespace cvf

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct cvf_handle {
  cvf_params p;
  long long N;
  cudaStream_t stream;
  cudaStream_t cap_stream;
  uint16_t* state;
  bool own_state;
  Ctrl* ctrl;
  cvf_obs* ring;
  long long ring_cap;
  long long ring_tail;
  cvf_obs* obs_dev;
  unsigned long long* table_dev;     // [2][24] (dN_HB+1)*8 + dN_sigma+3
  bool cmp64;                        // some threshold is 0: compare in 64 bits
  long long sweep_host;              // steps enqueued so far: buffer sweep & 1 is current
  VolumeArgs* vol_dev;
  unsigned long long* rc_dev;
  void* host_pinned;
  LatticeArgs args;
  CUtensorMap tm[2];  // TMA descriptors of the two halves of the state pair
  int grid_tiles, grid_cells, grid_layer;
  bool programmatic;  // sweep launches overlap the previous step (grid fills the GPU)
  int tile;  // tile shape of the sweep (see TileShape)
  cudaGraphExec_t graph;
  int graph_steps;
  WaveHdr* wave;  // scratch of the wavefront sweep (allocated when first chosen)
  size_t wave_bytes;
};

namespace {

constexpr long long kRingCap = 65536;
constexpr int kGraphSteps = 32;

int grid_for(long long work, int per_sm) {
  const long long blocks = (work + kThreads - 1) / kThreads;
  const long long cap = (long long)sm_count() * per_sm;
  return (int)std::max<long long>(1, std::min(blocks, cap));
}

void release(cvf_handle* h) {
  if (!h) return;
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->wave) cudaFree(h->wave);
  if (h->own_state && h->state) cudaFree(h->state);
  if (h->ctrl) cudaFree(h->ctrl);
  if (h->ring) cudaFree(h->ring);
  if (h->obs_dev) cudaFree(h->obs_dev);
  if (h->table_dev) cudaFree(h->table_dev);
  if (h->vol_dev) cudaFree(h->vol_dev);
  if (h->rc_dev) cudaFree(h->rc_dev);
  if (h->host_pinned) cudaFreeHost(h->host_pinned);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  delete h;
}

// Whether every tile of shape `tile` on an L x L lattice is full with rows
// 16-byte aligned (the column-walking form of the sweep).
template <int TILE>
bool walk_fits_t(int L) {
  return L % TileShape<TILE>::R == 0 && (L / 2) % TileShape<TILE>::W == 0 && (L / 2) % 4 == 0;
}

// The sweep kernel for (rng_words, cmp64, tile shape, lattice side).
template <int TILE, bool WALK>
const void* sweep_kernel_tw(int rng_words, bool cmp64) {
  if (rng_words == 1)
    return cmp64 ? (const void*)k_sweep_tiled<1, true, TILE, WALK>
                 : (const void*)k_sweep_tiled<1, false, TILE, WALK>;
  return cmp64 ? (const void*)k_sweep_tiled<2, true, TILE, WALK>
               : (const void*)k_sweep_tiled<2, false, TILE, WALK>;
}

template <int TILE>
const void* sweep_kernel_t(int rng_words, bool cmp64, int L) {
  return walk_fits_t<TILE>(L) ? sweep_kernel_tw<TILE, true>(rng_words, cmp64)
                              : sweep_kernel_tw<TILE, false>(rng_words, cmp64);
}

const void* sweep_kernel(int rng_words, bool cmp64, int tile, int L) {
  if (tile == 0) return sweep_kernel_t<0>(rng_words, cmp64, L);
  if (tile == 1) return sweep_kernel_t<1>(rng_words, cmp64, L);
  return sweep_kernel_t<2>(rng_words, cmp64, L);
}

cudaError_t launch_sweep(const void* fn, int grid, cudaStream_t s, const LatticeArgs& A,
                         const CUtensorMap& tm0, const CUtensorMap& tm1, bool programmatic) {
  void* args[3] = {const_cast<LatticeArgs*>(&A), const_cast<CUtensorMap*>(&tm0),
                   const_cast<CUtensorMap*>(&tm1)};
  // programmatic stream serialization: the launch overlaps the previous
  // step's tail; the kernel waits for that step before touching memory.
  // Used only when the grid fills every resident block slot: with a smaller
  // grid the next step's blocks take free slots early, unevenly (768^2, 577
  // of 760 slots: 13.1 against 11.8 us per step)
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = programmatic ? 1 : 0;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

// Enqueue one MC step on stream s; returns the launch error, if any.
cudaError_t enqueue_step(cvf_handle* h, cudaStream_t s) {
  const bool one = h->p.rng_words == 1;
  if (h->p.schedule == CVF_SCHED_CHECKERBOARD) {
    return launch_sweep(sweep_kernel(h->p.rng_words, h->cmp64, h->tile, h->p.L), h->grid_tiles, s,
                        h->args, h->tm[0], h->tm[1], h->programmatic);
  } else {
    for (int j = 0; j < kLayerLaunches; ++j) {
      const int grid = h->grid_layer + (j == 0 ? 1 : 0);  // + the volume block
      if (one && !h->cmp64)
        k_layer<1, false><<<grid, kThreads, 0, s>>>(h->args, j);
      else if (one)
        k_layer<1, true><<<grid, kThreads, 0, s>>>(h->args, j);
      else if (!h->cmp64)
        k_layer<2, false><<<grid, kThreads, 0, s>>>(h->args, j);
      else
        k_layer<2, true><<<grid, kThreads, 0, s>>>(h->args, j);
    }
    return cudaGetLastError();
  }
}

// The half of the state pair that holds the lattice after the enqueued steps.
uint16_t* current(cvf_handle* h) { return h->state + (size_t)(h->sweep_host & 1) * h->N; }

// TMA descriptors of the two lattice buffers (uint32 words, Lh x L, box of
// tile words + 8 x tile rows + 4).  Needs 16-byte aligned rows and buffers
// (L a multiple of 8); returns false (cp.async staging only) when that or
// the driver entry point is unavailable.
bool encode_state_maps(uint16_t* state, int L, int tile_rows, int tile_words, CUtensorMap tm[2]) {
  std::memset(tm, 0, sizeof(CUtensorMap) * 2);
  if (L % 8 != 0) return false;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return false;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const long long N = (long long)L * L;
  const cuuint64_t dims[2] = {(cuuint64_t)(L / 2), (cuuint64_t)L};
  const cuuint64_t strides[1] = {(cuuint64_t)(L / 2) * 4};
  const cuuint32_t box[2] = {(cuuint32_t)tile_words + 8, (cuuint32_t)tile_rows + 4};
  const cuuint32_t elem[2] = {1, 1};
  for (int b = 0; b < 2; ++b) {
    void* base = state + (size_t)b * N;
    if (reinterpret_cast<uintptr_t>(base) & 15u) return false;
    if (encode(&tm[b], CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, base, dims, strides, box, elem,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
        CUDA_SUCCESS)
      return false;
  }
  return true;
}

// Tile config kResident: the whole lattice resident in one cluster's shared
// memory (cvf_resident2.cu), one slab of L / kResCtas rows per CTA.
constexpr int kResident = kNumSweepTiles;
// Tile configs kWave + shape: the wavefront sweep (cvf_wave.cu) on the tile
// shapes 0 .. kNumSweepTiles - 1.
constexpr int kWave = kResident + 1;
constexpr int kMaxTileConfig = kWave + kNumSweepTiles - 1;
bool is_wave(int tile) { return tile >= kWave; }
// the automatic choice takes the resident sweep up to this side (measured:
// it beats the tiled sweep there)
constexpr int kResAutoSide = 128;

void tile_shape(int tile, int L, int* rows, int* words) {
  if (tile == kResident) {
    *rows = L / kResCtas;
    *words = L / 2;
    return;
  }
  if (is_wave(tile)) tile -= kWave;
  *rows = (tile == 0) ? TileShape<0>::R : (tile == 1) ? TileShape<1>::R : TileShape<2>::R;
  *words = (tile == 0) ? TileShape<0>::W : (tile == 1) ? TileShape<1>::W : TileShape<2>::W;
}

long long tile_count(int L, int tile) {
  int r, w;
  tile_shape(tile, L, &r, &w);
  return (long long)((L / 2 + w - 1) / w) * ((L + r - 1) / r);
}

int resident_sweep_blocks(bool cmp64, int rng_words, int tile) {
  int per_sm = 1;
  // (both forms of the kernel have the same registers and shared memory)
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel(rng_words, cmp64, tile, 1),
                                                    kThreads, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return sm_count() * per_sm;
}

// Tile shape for a lattice: the largest whose tiles fill every resident
// block, else the smallest.
int choose_tile(int L, bool cmp64, int rng_words) {
  for (int t = 0; t < kNumSweepTiles; ++t)
    if (tile_count(L, t) >= resident_sweep_blocks(cmp64, rng_words, t)) return t;
  return kNumSweepTiles - 1;
}

// Persistent grid of the tiled sweep: as many blocks as fit on the GPU at
// once, but no more than there are tiles.
int tiled_grid(int L, bool cmp64, int rng_words, int tile) {
  const long long tiles = tile_count(L, tile);
  const long long resident = resident_sweep_blocks(cmp64, rng_words, tile);
  // + 1: block 0 decides the next volume move instead of taking tiles
  return 1 + (int)std::max<long long>(1, std::min<long long>(tiles, resident));
}

// The wavefront sweep needs the checkerboard schedule, rows on 16-byte
// boundaries (L a multiple of 8) and at least 3 x 3 tiles (every tile's
// neighbourhood then holds the rows and words its halo reads).
bool wave_fits(const cvf_handle* h, int shape) {
  if (h->p.schedule != CVF_SCHED_CHECKERBOARD || h->p.L % 8 != 0) return false;
  int r, w;
  tile_shape(shape, h->p.L, &r, &w);
  const int tx = (h->p.L / 2 + w - 1) / w, ty = (h->p.L + r - 1) / r;
  return tx >= 3 && ty >= 3 && wave_blocks(h->p.rng_words, h->cmp64, shape) >= 2;
}

// Scratch of the wavefront sweep for tile shape `shape`.
int wave_scratch(cvf_handle* h, int shape) {
  int r, w;
  tile_shape(shape, h->p.L, &r, &w);
  const long long tiles = (long long)((h->p.L / 2 + w - 1) / w) * ((h->p.L + r - 1) / r);
  const size_t bytes = sizeof(WaveHdr) + sizeof(unsigned int) * (size_t)tiles;
  if (h->wave && h->wave_bytes >= bytes) return CVF_OK;
  if (h->wave) cudaFree(h->wave);
  h->wave = nullptr;
  h->wave_bytes = 0;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&h->wave), bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(e == cudaErrorMemoryAllocation ? CVF_ENOMEM : CVF_ECUDA,
                     "wavefront scratch (%zu bytes): %s", bytes, cudaGetErrorString(e));
  }
  h->wave_bytes = bytes;
  return CVF_OK;
}

// The automatic configuration: the resident form for small lattices; the
// wavefront sweep from 256^2 up, with the tiled sweep's shape rule (the
// largest shape with at least as many tiles as the tiled sweep has resident
// blocks: the fastest wavefront shape at 768^2, 1536^2, 2048^2 and from
// 2560^2 up, within 1.2 % of it at 1024^2, where 32 x 32 words ran at 11.2
// against 11.3 us per step); the tiled sweep with that shape where the
// wavefront does not fit.
// Measured on GB300, us per MC step, wavefront against the best tiled shape:
// 256^2 6.6 / 7.5, 320^2 6.4 / 7.5, 384^2 7.0 / 7.4, 448^2 7.3 / 8.1,
// 512^2 7.6 / 8.3, 1024^2 11.3 / 14.3, 2048^2 31.8 / 36.8, 3072^2 61.8 /
// 71.3, 4096^2 103.0 / 115.0, 6144^2 226.6 / 248.9, 8192^2 402.3 / 428.5,
// 12288^2 902.9 / 941.6, 16384^2 1603.5 / 1656.9 (the tiled sweep's partly
// filled last round of tiles costs less the more tiles a step has, but the
// wavefront stays ahead).
constexpr int kWaveAutoMin = 256;
int auto_config(const cvf_handle* h) {
  const cvf_params& p = h->p;
  if (p.schedule == CVF_SCHED_CHECKERBOARD && p.L <= kResAutoSide &&
      resident_fits(h->args, p.rng_words, h->cmp64))
    return kResident;
  const int t = choose_tile(p.L, h->cmp64, p.rng_words);
  if (p.L >= kWaveAutoMin && wave_fits(h, t)) return kWave + t;
  return t;
}

// Adopt tile shape `tile` for the handle: grid, TMA boxes, and a new graph.
void set_tile(cvf_handle* h, int tile) {
  h->tile = tile;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
  if (tile == kResident) return;
  int r, w;
  tile_shape(tile, h->p.L, &r, &w);
  if (is_wave(tile)) {  // the wavefront stages interior tiles with these boxes too
    h->args.use_tma = encode_state_maps(h->state, h->p.L, r, w, h->tm) ? 1 : 0;
    return;
  }
  h->grid_tiles = tiled_grid(h->p.L, h->cmp64, h->p.rng_words, tile);
  h->programmatic =
      tile_count(h->p.L, tile) >= resident_sweep_blocks(h->cmp64, h->p.rng_words, tile);
  h->args.use_tma = encode_state_maps(h->state, h->p.L, r, w, h->tm) ? 1 : 0;
  if (h->graph) {
    cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
  }
}

int recount_into_ctrl(cvf_handle* h) {
  // acc_hb and acc_pairs are adjacent: the recount adds into both
  static_assert(offsetof(Ctrl, acc_pairs) == offsetof(Ctrl, acc_hb) + 8, "layout");
  k_recount<<<h->grid_cells, kThreads, 0, h->stream>>>(current(h), h->p.L, nullptr,
                                                       &h->ctrl->acc_hb);
  k_commit_counts<<<1, 32, 0, h->stream>>>(h->ctrl);
  k_volume_prologue<<<1, 32, 0, h->stream>>>(h->vol_dev, h->ctrl, h->args.keys);
  CVF_CUDA_CHECK(cudaGetLastError());
  return CVF_OK;
}

// Index of the first word that is not a valid cell (a nibble >= q, or a
// nibble's bit 3 set), n if none.  Four cells per 64-bit load: with the
// guard bits clear every nibble v is <= 7, and v + 8 - q sets the nibble's
// bit 3 exactly when v >= q (no carry leaves a nibble: v + 8 - q <= 13).
int build_graph(cvf_handle* h) {
  if (h->graph) return CVF_OK;
  cudaGraph_t g = nullptr;
  CVF_CUDA_CHECK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  for (int i = 0; i < kGraphSteps && le == cudaSuccess; ++i) le = enqueue_step(h, h->cap_stream);
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return set_error(CVF_ECUDA, "graph capture: launch failed: %s", cudaGetErrorString(le));
  }
  if (e != cudaSuccess) return set_error(CVF_ECUDA, "graph capture: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->graph = nullptr;
    return set_error(CVF_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  h->graph_steps = kGraphSteps;
  return CVF_OK;
}

}  // namespace

extern "C" {

int cvf_create(const cvf_params* p, void* stream, void* dev_state, cvf_handle** out) {
  NvtxRange nvtx_range("cvf_create");
  if (!out) return set_error(CVF_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = check_params(p);
  if (rc) return rc;
  if (dev_state && (reinterpret_cast<uintptr_t>(dev_state) & 15u))
    return set_error(CVF_EINVAL, "dev_state must be 16-byte aligned");
  std::vector<int64_t> d2, mult;
  lattice_shells(p->cutoff, &d2, &mult);
  if ((int)d2.size() > kMaxShells)
    return set_error(CVF_EINVAL, "cutoff %g needs %zu shells (max %d)", p->cutoff, d2.size(),
                     kMaxShells);
  cvf_handle* h = new (std::nothrow) cvf_handle();
  if (!h) return set_error(CVF_ENOMEM, "host allocation failed");
  std::memset(h, 0, sizeof(*h));
  h->p = *p;
  h->N = (long long)p->L * p->L;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  h->ring_cap = kRingCap;
#define CREATE_CHECK(expr)                                                        \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess) {                                                      \
      int code_ = (e_ == cudaErrorMemoryAllocation) ? CVF_ENOMEM : CVF_ECUDA;     \
      set_error(code_, "%s failed: %s", #expr, cudaGetErrorString(e_));           \
      release(h);                                                                 \
      return code_;                                                               \
    }                                                                             \
  } while (0)
  CREATE_CHECK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  if (dev_state) {
    h->state = reinterpret_cast<uint16_t*>(dev_state);
    h->own_state = false;
  } else {
    CREATE_CHECK(cudaMalloc(&h->state, sizeof(uint16_t) * 2 * (size_t)h->N));
    h->own_state = true;
  }
  CREATE_CHECK(cudaMalloc(&h->ctrl, sizeof(Ctrl)));
  CREATE_CHECK(cudaMalloc(&h->ring, sizeof(cvf_obs) * (size_t)h->ring_cap));
  CREATE_CHECK(cudaMalloc(&h->obs_dev, sizeof(cvf_obs)));
  CREATE_CHECK(cudaMalloc(&h->table_dev, sizeof(unsigned long long) * 48));
  CREATE_CHECK(cudaMalloc(&h->vol_dev, sizeof(VolumeArgs)));
  CREATE_CHECK(cudaMalloc(&h->rc_dev, sizeof(unsigned long long) * 9));
  CREATE_CHECK(cudaMallocHost(&h->host_pinned, 4096));

  unsigned long long table24[48];
  h->cmp64 = fill_table24(p, table24);
  VolumeArgs va;
  fill_volume_args(p, h->N, d2, mult, &va);
  CREATE_CHECK(cudaMemcpyAsync(h->table_dev, table24, sizeof(table24), cudaMemcpyHostToDevice,
                               h->stream));
  CREATE_CHECK(cudaMemcpyAsync(h->vol_dev, &va, sizeof(va), cudaMemcpyHostToDevice, h->stream));
  CREATE_CHECK(cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));

  h->args.state = h->state;
  h->args.ctrl = h->ctrl;
  h->args.table24 = h->table_dev;
  h->args.vol = h->vol_dev;
  h->args.ring = h->ring;
  h->args.ring_cap = h->ring_cap;
  h->args.keys = make_round_keys(p->seed);
  h->args.L = p->L;
  h->args.q = (uint32_t)p->q;
  {
    const int cfg = auto_config(h);
    if (is_wave(cfg)) {
      rc = wave_scratch(h, cfg - kWave);
      if (rc) {
        release(h);
        return rc;
      }
    }
    set_tile(h, cfg);
  }
  h->sweep_host = 0;
  h->grid_cells = grid_for(h->N, 8);
  h->grid_layer = grid_for(h->N / 2, 8);  // one word (two cells) per thread and iteration

  k_init<<<h->grid_cells, kThreads, 0, h->stream>>>(h->state, p->L, (uint32_t)p->q,
                                                     p->init == CVF_INIT_RANDOM ? 1 : 0,
                                                     h->args.keys);
  k_set_ctrl<<<1, 32, 0, h->stream>>>(h->vol_dev, h->ctrl, (double)h->N * p->v_iso_init, 0,
                                      h->N);
  rc = recount_into_ctrl(h);
  if (rc) {
    release(h);
    return rc;
  }
  CREATE_CHECK(cudaGetLastError());
  CREATE_CHECK(cudaStreamSynchronize(h->stream));
#undef CREATE_CHECK
  *out = h;
  return CVF_OK;
}

int cvf_sweep(cvf_handle* h, int64_t n_sweeps, int32_t record_every) {
  NvtxRange nvtx_range("cvf_sweep");
  if (!h) return set_error(CVF_EINVAL, "handle is NULL");
  if (n_sweeps < 0 || record_every < 0)
    return set_error(CVF_EINVAL, "n_sweeps=%lld, record_every=%d must be >= 0",
                     (long long)n_sweeps, record_every);
  if (n_sweeps == 0) return CVF_OK;
  k_set_record<<<1, 32, 0, h->stream>>>(h->ctrl, record_every);
  if (is_wave(h->tile)) {
    // one persistent launch per 2^30 steps (the launch's step counters are 32-bit)
    constexpr long long kChunk = 1ll << 30;
    for (long long done = 0; done < n_sweeps; done += kChunk)
      CVF_CUDA_CHECK(launch_wave(h->args, h->wave, h->wave_bytes, h->p.rng_words, h->cmp64,
                                 h->tile - kWave, h->sweep_host + done,
                                 std::min(kChunk, n_sweeps - done), h->tm, h->stream));
    h->sweep_host += n_sweeps;
    return CVF_OK;
  }
  if (h->tile == kResident && h->p.schedule == CVF_SCHED_CHECKERBOARD) {
    // many steps per launch; the lattice stays in the cluster's shared memory
    constexpr long long kChunk = 1 << 16;
    for (long long done = 0; done < n_sweeps; done += kChunk)
      CVF_CUDA_CHECK(launch_resident(h->args, h->p.rng_words, h->cmp64,
                                     std::min(kChunk, n_sweeps - done), h->stream));
    h->sweep_host += n_sweeps;
    return CVF_OK;
  }
  long long left = n_sweeps;
  if (left >= kGraphSteps) {
    int rc = build_graph(h);
    if (rc) return rc;
    while (left >= h->graph_steps) {
      CVF_CUDA_CHECK(cudaGraphLaunch(h->graph, h->stream));
      left -= h->graph_steps;
    }
  }
  for (; left > 0; --left) CVF_CUDA_CHECK(enqueue_step(h, h->stream));
  CVF_CUDA_CHECK(cudaGetLastError());
  h->sweep_host += n_sweeps;
  return CVF_OK;
}

int cvf_observables(cvf_handle* h, cvf_obs* out) {
  NvtxRange nvtx_range("cvf_observables");
  if (!h || !out) return set_error(CVF_EINVAL, "NULL argument");
  CVF_CUDA_CHECK(cudaMemsetAsync(h->rc_dev, 0, sizeof(unsigned long long) * 9, h->stream));
  k_histogram<<<h->grid_cells, kThreads, 0, h->stream>>>(current(h), h->N, h->rc_dev);
  k_observables<<<1, 32, 0, h->stream>>>(h->vol_dev, h->ctrl, h->rc_dev, h->obs_dev);
  CVF_CUDA_CHECK(cudaGetLastError());
  CVF_CUDA_CHECK(cudaMemcpyAsync(h->host_pinned, h->obs_dev, sizeof(cvf_obs),
                                 cudaMemcpyDeviceToHost, h->stream));
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  std::memcpy(out, h->host_pinned, sizeof(cvf_obs));
  return status_error(out->status);
}

int cvf_drain_series(cvf_handle* h, cvf_obs* host, int64_t cap, int64_t* n) {
  NvtxRange nvtx_range("cvf_drain_series");
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
  long long avail = c.ring_head - h->ring_tail;
  long long take = std::min<long long>(avail, cap);
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

int cvf_get_state(cvf_handle* h, uint16_t* host, size_t n) {
  NvtxRange nvtx_range("cvf_get_state");
  if (!h || !host) return set_error(CVF_EINVAL, "NULL argument");
  if ((long long)n != h->N) return set_error(CVF_EINVAL, "n=%zu, lattice has %lld cells", n, h->N);
  CVF_CUDA_CHECK(cudaMemcpyAsync(host, current(h), sizeof(uint16_t) * n, cudaMemcpyDeviceToHost,
                                 h->stream));
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  return CVF_OK;
}

int cvf_get_window(cvf_handle* h, int32_t x0, int32_t y0, int32_t W, int32_t H,
                   uint16_t* host) {
  NvtxRange nvtx_range("cvf_get_window");
  if (!h || !host) return set_error(CVF_EINVAL, "NULL argument");
  const long long L = h->p.L;
  if (W < 1 || H < 1 || x0 < 0 || y0 < 0 || (long long)x0 + W > L || (long long)y0 + H > L)
    return set_error(CVF_EINVAL, "window x0=%d y0=%d W=%d H=%d outside the %lld x %lld lattice",
                     x0, y0, W, H, L, L);
  const uint16_t* src = current(h) + (size_t)y0 * (size_t)L + (size_t)x0;
  CVF_CUDA_CHECK(cudaMemcpy2DAsync(host, sizeof(uint16_t) * (size_t)W, src,
                                   sizeof(uint16_t) * (size_t)L, sizeof(uint16_t) * (size_t)W,
                                   (size_t)H, cudaMemcpyDeviceToHost, h->stream));
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  return CVF_OK;
}

int cvf_set_state(cvf_handle* h, const uint16_t* host, size_t n, double V_iso, int64_t sweep) {
  NvtxRange nvtx_range("cvf_set_state");
  if (!h || !host) return set_error(CVF_EINVAL, "NULL argument");
  if ((long long)n != h->N) return set_error(CVF_EINVAL, "n=%zu, lattice has %lld cells", n, h->N);
  if (!(V_iso >= (double)h->N) || !std::isfinite(V_iso))
    return set_error(CVF_EINVAL, "V_iso=%g below the hard core N v0 = %lld", V_iso, h->N);
  if (sweep < 0) return set_error(CVF_EINVAL, "sweep must be >= 0");
  // The words go to the state pair's other buffer (free between calls) and
  // are checked there on the device; only a valid lattice replaces the
  // current one (a device copy where the new step parity needs the other
  // buffer), so an invalid upload leaves the handle as it was.
  const size_t bytes = sizeof(uint16_t) * n;
  uint16_t* up = h->state + (size_t)((h->sweep_host + 1) & 1) * h->N;
  CVF_CUDA_CHECK(cudaMemcpyAsync(up, host, bytes, cudaMemcpyHostToDevice, h->stream));
  CVF_CUDA_CHECK(cudaMemsetAsync(h->rc_dev, 0xFF, sizeof(unsigned long long), h->stream));
  k_first_invalid<<<h->grid_cells, kThreads, 0, h->stream>>>(up, h->N, (uint32_t)h->p.q,
                                                              h->rc_dev);
  CVF_CUDA_CHECK(cudaGetLastError());
  CVF_CUDA_CHECK(cudaMemcpyAsync(h->host_pinned, h->rc_dev, sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, h->stream));
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  const unsigned long long bad = *reinterpret_cast<const unsigned long long*>(h->host_pinned);
  if (bad < (unsigned long long)n)
    return set_error(CVF_EINVAL, "word %llu = 0x%04x is not a valid cell for q = %d", bad,
                     (unsigned)host[bad], h->p.q);
  uint16_t* dst = h->state + (size_t)(sweep & 1) * h->N;
  if (dst != up)
    CVF_CUDA_CHECK(cudaMemcpyAsync(dst, up, bytes, cudaMemcpyDeviceToDevice, h->stream));
  h->sweep_host = sweep;
  k_set_ctrl<<<1, 32, 0, h->stream>>>(h->vol_dev, h->ctrl, V_iso, sweep, h->N);
  int rc = recount_into_ctrl(h);
  if (rc) return rc;
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  h->ring_tail = 0;
  return CVF_OK;
}

int cvf_recount(cvf_handle* h, int64_t* n_hb_raw, int64_t* n_sigma) {
  NvtxRange nvtx_range("cvf_recount");
  if (!h || !n_hb_raw || !n_sigma) return set_error(CVF_EINVAL, "NULL argument");
  CVF_CUDA_CHECK(cudaMemsetAsync(h->rc_dev, 0, sizeof(unsigned long long) * 2, h->stream));
  k_recount<<<h->grid_cells, kThreads, 0, h->stream>>>(current(h), h->p.L, nullptr, h->rc_dev);
  CVF_CUDA_CHECK(cudaGetLastError());
  CVF_CUDA_CHECK(cudaMemcpyAsync(h->host_pinned, h->rc_dev, sizeof(unsigned long long) * 2,
                                 cudaMemcpyDeviceToHost, h->stream));
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  const unsigned long long* r = reinterpret_cast<const unsigned long long*>(h->host_pinned);
  *n_hb_raw = (int64_t)r[0];
  *n_sigma = (int64_t)r[1];
  return CVF_OK;
}

int cvf_state_device_ptr(cvf_handle* h, void** dev_ptr) {
  if (!h || !dev_ptr) return set_error(CVF_EINVAL, "NULL argument");
  *dev_ptr = current(h);
  return CVF_OK;
}

int cvf_set_tiles(cvf_handle* h, int32_t config) {
  if (!h) return set_error(CVF_EINVAL, "handle is NULL");
  if (config < -1 || config > kMaxTileConfig)
    return set_error(CVF_EINVAL, "tile config %d: need -1 (automatic) or 0..%d", config,
                     kMaxTileConfig);
  const bool res_ok = h->p.schedule == CVF_SCHED_CHECKERBOARD &&
                      resident_fits(h->args, h->p.rng_words, h->cmp64);
  if (config == kResident && !res_ok)
    return set_error(CVF_EINVAL, "the resident sweep needs the checkerboard schedule and "
                     "%d <= L <= %d, L a multiple of %d", 2 * kResCtas, kResMaxSide, kResCtas);
  if (is_wave(config) && !wave_fits(h, config - kWave))
    return set_error(CVF_EINVAL, "the wavefront sweep needs the checkerboard schedule, L a "
                     "multiple of 8 and at least 3 x 3 tiles of the shape");
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  if (is_wave(config)) {
    const int rc = wave_scratch(h, config - kWave);
    if (rc) return rc;
  }
  if (config < 0) config = auto_config(h);
  set_tile(h, config);
  return CVF_OK;
}

int cvf_get_tiles(cvf_handle* h, int32_t* config, int32_t* rows, int32_t* words) {
  if (!h || !config || !rows || !words) return set_error(CVF_EINVAL, "NULL argument");
  int r, w;
  tile_shape(h->tile, h->p.L, &r, &w);
  *config = h->tile;
  *rows = r;
  *words = w;
  return CVF_OK;
}

int cvf_destroy(cvf_handle* h) {
  if (!h) return CVF_OK;
  cudaError_t e = cudaStreamSynchronize(h->stream);
  release(h);
  if (e != cudaSuccess) return set_error(CVF_ECUDA, "destroy: %s", cudaGetErrorString(e));
  return CVF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free sweep (cvf_sweep_noalloc).  Everything the sweep needs
// besides the caller's lattice -- the control block with its counters, the
// threshold rows, the FP64 parameters and a short observable ring -- lives in
// one file-scope device array of fixed size instead of memory from
// cudaMalloc.  Every GPU that loads the library holds this array until the
// process exits.  All calls on a device share it: the call clears what must
// start at zero, and calls whose GPU work overlaps race on it.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocRing = 256;                 // recorded steps per call
constexpr size_t kNoAllocScratchBytes = 64 * 1024;

struct NoAllocScratch {
  Ctrl ctrl;
  unsigned long long hist[9];
  unsigned long long table24[48];
  VolumeArgs vol;
  cvf_obs obs;
  cvf_obs ring[kNoAllocRing];
};
static_assert(sizeof(NoAllocScratch) <= kNoAllocScratchBytes, "scratch layout");

struct Table48 {
  unsigned long long t[48];
};

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

namespace cvf {

// Flags (status bit kStatusBadCell in *err) a lattice holding a word that is
// not a valid cell for q: a guard bit set or a nibble >= q.  The caller's
// buffer is not checked on the host (that would need a copy).
__global__ void __launch_bounds__(kThreads) k_check_cells(const uint16_t* __restrict__ state,
                                                          long long N, uint32_t q,
                                                          unsigned int* err) {
  bool bad = false;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const uint32_t w = state[c];
    bad |= (w & 0x8888u) != 0u || (w & 7u) >= q || ((w >> 4) & 7u) >= q ||
           ((w >> 8) & 7u) >= q || ((w >> 12) & 7u) >= q;
  }
  if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31u) == 0u) atomicOr(err, kStatusBadCell);
}

// Copies the call's parameters (passed by value) into the scratch and clears
// the control block.
__global__ void k_noalloc_setup(NoAllocScratch* s, VolumeArgs va, Table48 t) {
  if (blockIdx.x != 0) return;
  for (int i = threadIdx.x; i < 48; i += blockDim.x) s->table24[i] = t.t[i];
  unsigned char* c = reinterpret_cast<unsigned char*>(&s->ctrl);
  for (int i = threadIdx.x; i < (int)sizeof(Ctrl); i += blockDim.x) c[i] = 0;
  if (threadIdx.x == 0) s->vol = va;
}

}  // namespace cvf

namespace {

// Device address of the scratch array on the current device, looked up on
// every call (host code may not use the array's name as a device address;
// the lookup is cheap, and a context torn down and rebuilt -- a device
// reset -- may place the array elsewhere, so no address is kept).
int noalloc_scratch(NoAllocScratch** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || !ptr)
    return set_error(CVF_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s",
                     cudaGetErrorString(e));
  *out = reinterpret_cast<NoAllocScratch*>(ptr);
  return CVF_OK;
}

// The FP64 parameters and LJ shell prefix sums, built in fixed-size storage
// (this path allocates nothing, not even host memory).  Same shells, same
// order, same sums as fill_volume_args.
int noalloc_volume_args(const cvf_params* p, long long N, VolumeArgs* va) {
  std::memset(va, 0, sizeof(*va));
  const int R = (int)std::ceil(p->cutoff);
  int n = 0;
  va->S12[0] = 0.0;
  va->S6[0] = 0.0;
  for (int64_t d2 = 1; d2 <= 2LL * R * R; ++d2) {
    int64_t m = 0;
    for (int i = -R; i <= R; ++i)
      for (int j = -R; j <= R; ++j)
        if ((int64_t)i * i + (int64_t)j * j == d2) ++m;
    if (m == 0 || !((double)d2 < p->cutoff * p->cutoff)) continue;
    if (n >= kMaxShells) return set_error(CVF_EINVAL, "cutoff too large");
    va->shell_d2[n] = (double)d2;
    const int64_t d6 = d2 * d2 * d2;
    va->S12[n + 1] = va->S12[n] + (double)m / ((double)d6 * (double)d6);
    va->S6[n + 1] = va->S6[n] + (double)m / (double)d6;
    ++n;
  }
  va->nshell = n;
  va->N = N;
  va->epsilon = p->epsilon;
  va->cutoff2 = p->cutoff * p->cutoff;
  va->J = p->J;
  va->J_sigma = p->J_sigma;
  va->v_HB = p->v_HB;
  va->kT = p->kT;
  va->P = p->P;
  va->dV_max = p->dv_max_frac * ((double)N * p->v_iso_init);
  va->volume_moves = p->volume_moves;
  return CVF_OK;
}

}  // namespace

extern "C" int cvf_sweep_noalloc(const cvf_params* p, void* dev_state, double V_iso,
                                 int64_t sweep, int64_t n_sweeps, int32_t record_every,
                                 cvf_obs* host_series, int64_t series_cap, int64_t* n_series,
                                 cvf_obs* host_obs, void* stream) {
  int rc = check_params(p);
  if (rc) return rc;
  if (!dev_state || !host_obs || !n_series)
    return set_error(CVF_EINVAL, "dev_state, host_obs and n_series are required");
  if (reinterpret_cast<uintptr_t>(dev_state) & 15u)
    return set_error(CVF_EINVAL, "dev_state must be 16-byte aligned");
  if (p->schedule != CVF_SCHED_CHECKERBOARD)
    return set_error(CVF_EINVAL, "cvf_sweep_noalloc runs the checkerboard schedule only");
  const long long N = (long long)p->L * p->L;
  if (!(V_iso >= (double)N) || !std::isfinite(V_iso))
    return set_error(CVF_EINVAL, "V_iso=%g below the hard core N v0 = %lld", V_iso, N);
  if (sweep < 0 || n_sweeps < 0 || record_every < 0 || series_cap < 0)
    return set_error(CVF_EINVAL, "sweep, n_sweeps, record_every and series_cap must be >= 0");
  long long records = 0;
  if (record_every > 0)
    records = (sweep + n_sweeps) / record_every - sweep / record_every;
  if (records > kNoAllocRing)
    return set_error(CVF_EINVAL,
                     "%lld recorded steps requested; this entry point keeps at most %d per call",
                     records, kNoAllocRing);
  if (records > series_cap || (records > 0 && !host_series))
    return set_error(CVF_EINVAL, "host_series holds %lld records, %lld needed",
                     (long long)series_cap, records);
  NoAllocScratch* s = nullptr;
  rc = noalloc_scratch(&s);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Table48 t48;
  const bool cmp64 = fill_table24(p, t48.t);
  VolumeArgs va;
  rc = noalloc_volume_args(p, N, &va);
  if (rc) return rc;
  LatticeArgs A;
  std::memset(&A, 0, sizeof(A));
  A.state = reinterpret_cast<uint16_t*>(dev_state);
  A.ctrl = &s->ctrl;
  A.table24 = s->table24;
  A.vol = &s->vol;
  A.ring = s->ring;
  A.ring_cap = kNoAllocRing;
  A.keys = make_round_keys(p->seed);
  A.L = p->L;
  A.q = (uint32_t)p->q;
  uint16_t* cur = A.state + (size_t)(sweep & 1) * N;
  const int grid_cells = grid_for(N, 8);
  k_noalloc_setup<<<1, 256, 0, st>>>(s, va, t48);
  k_check_cells<<<grid_cells, kThreads, 0, st>>>(cur, N, A.q, &s->ctrl.error);
  k_set_ctrl<<<1, 32, 0, st>>>(&s->vol, &s->ctrl, V_iso, sweep, N);
  k_recount<<<grid_cells, kThreads, 0, st>>>(cur, p->L, nullptr, &s->ctrl.acc_hb);
  k_commit_counts<<<1, 32, 0, st>>>(&s->ctrl);
  k_volume_prologue<<<1, 32, 0, st>>>(&s->vol, &s->ctrl, A.keys);
  k_set_record<<<1, 32, 0, st>>>(&s->ctrl, record_every);
  const int tile = choose_tile(p->L, cmp64, p->rng_words);
  const int grid = tiled_grid(p->L, cmp64, p->rng_words, tile);
  const void* fn = sweep_kernel(p->rng_words, cmp64, tile, p->L);
  CUtensorMap no_map;  // this path stages every tile with cp.async
  std::memset(&no_map, 0, sizeof(no_map));
  const bool programmatic =
      tile_count(p->L, tile) >= resident_sweep_blocks(cmp64, p->rng_words, tile);
  for (int64_t i = 0; i < n_sweeps; ++i)
    CVF_CUDA_CHECK(launch_sweep(fn, grid, st, A, no_map, no_map, programmatic));
  CVF_CUDA_CHECK(cudaMemsetAsync(s->hist, 0, sizeof(s->hist), st));
  k_histogram<<<grid_cells, kThreads, 0, st>>>(A.state + (size_t)((sweep + n_sweeps) & 1) * N, N,
                                               s->hist);
  k_observables<<<1, 32, 0, st>>>(&s->vol, &s->ctrl, s->hist, &s->obs);
  CVF_CUDA_CHECK(cudaGetLastError());
  CVF_CUDA_CHECK(cudaMemcpyAsync(host_obs, &s->obs, sizeof(cvf_obs), cudaMemcpyDeviceToHost, st));
  if (records > 0)
    CVF_CUDA_CHECK(cudaMemcpyAsync(host_series, s->ring, sizeof(cvf_obs) * records,
                                   cudaMemcpyDeviceToHost, st));
  CVF_CUDA_CHECK(cudaStreamSynchronize(st));
  *n_series = records;
  // a bounded wait that gave up, a failed index check of a debug build, or a
  // caller lattice holding an invalid cell
  return status_error(host_obs->status);
}
