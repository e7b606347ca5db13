// cvf_wave.cu -- the checkerboard sweep of one square lattice as a single
// persistent, cooperative launch per call, without a grid-wide barrier
// between MC steps (a wavefront).
//
// Work items are (relative step r, tile t), taken from one counter in
// step-major order.  A tile of step r reads its own cells and a halo of two
// rows and one word from the tiles around it, as they are after step r - 1,
// and writes the other buffer of the state pair; so item (r, t) waits only
// until the 3 x 3 tiles around t have finished step r - 1 (per-tile progress
// words, release / acquire).  That one condition also keeps a tile from
// overwriting words that a neighbour of the step before still has to read
// (the neighbourhood is symmetric).  The gate of step r comes from the volume
// move of step r, which block 0 decides ahead for every step from the move
// before it (Sec. II.B step 1: no bonds are needed unless the proposal would
// change the gate; then it waits for the commit of step r - 1 and decides
// with its N_HB).  Each tile adds its counts to its step's accumulators; the
// tile that completes a step commits it (counts, the step's volume move, the
// observables record), strictly in step order.  At most kWaveRing steps are
// in flight: a tile of step r also waits until step r - kWaveRing is
// committed, so the per-step slots can be reused.
//
// Items are processed in counter order by co-resident blocks (a cooperative
// launch), and every wait is for earlier items or for the engine, which
// waits only for commits of earlier steps: the oldest unfinished item can
// always run.  Every wait is bounded; one that gives up sets the lattice's
// error bit and the abort word, and every block then stops (CVF_ETIMEOUT).
// Each cell is updated by the same update_in_word with the same draws as in
// the tiled sweep, so the lattice, the counts and the records are the same.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "cvf_device.cuh"
#include "cvf_fastdiv.cuh"
#include "cvf_host.h"
#include "cvf_lattice.cuh"
#include "cvf_tile.cuh"
#include "cvf_tma.cuh"

namespace cvf {
namespace {

constexpr int kWaveShape = kHalfRows | kUnroll1 | kSplitRec;  // the tiled sweep's loops

// The tile grid of a launch, with the divisions it needs precomputed.
struct WaveGeom {
  int tiles_x, tiles_y, T;  // tiles per row, per column, per step
  FastDiv div_T, div_x;     // item -> (step, tile); tile -> (row, column)
  int small;                // the call's item count fits 32 bits
};

// Item i -> (relative step, tile).
__device__ __forceinline__ void wave_item(const WaveGeom& G, unsigned long long i, int* r,
                                          int* t) {
  if (G.small) {
    const uint32_t q = fdiv((uint32_t)i, G.div_T);
    *r = (int)q;
    *t = (int)((uint32_t)i - q * (uint32_t)G.T);
  } else {
    const long long q = (long long)(i / (unsigned long long)G.T);
    *r = (int)q;
    *t = (int)((long long)i - q * G.T);
  }
}
constexpr int kWaveEngineBar = 5;                             // the engine's two warps
// Bounded wait for a TMA stage (the copies complete in microseconds; the
// limit only guards against a copy that never lands).
constexpr uint32_t kWaveTmaWaitLimit = 1u << 26;

__device__ __forceinline__ void st_release_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}

__device__ __forceinline__ void st_relaxed_u32(unsigned int* p, unsigned int v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned int atom_add_relaxed_u32(unsigned int* p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.relaxed.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v)
               : "memory");
  return old;
}

__device__ __forceinline__ void engine_sync() {
  asm volatile("bar.sync %0, 64;" ::"n"(kWaveEngineBar) : "memory");
}

// Bounded wait of one thread until *flag >= target (or the launch aborts);
// false when it gave up or saw the abort word.
__device__ bool wave_wait_geq(const unsigned int* flag, unsigned int target, WaveHdr* H,
                              unsigned int* err) {
  unsigned int used = 0;
  for (;;) {
    if (ld_acquire(flag) >= target) return true;
    if (*(volatile unsigned int*)&H->abort) return false;
    used += 1;
    if (used > kWaitPollLimit) {
      atomicOr(err, 1u);
      atomicExch(&H->abort, 1u);
      return false;
    }
    __nanosleep(128);
  }
}

// The dependencies of item (r, t), tested by one warp: lanes 0..8 the nine
// tiles around t (progress >= r), lane 9 the step's volume move (published),
// lane 10 the commit of step r - kWaveRing (its slots are free).  With
// `block`, waits (bounded) until all hold; returns whether they hold (false
// also on an abort).  The move's gate is returned in *g (lane 0).
__device__ bool wave_deps(WaveHdr* H, const unsigned int* prog, int r, int t, const WaveGeom& G,
                          bool block, unsigned int* err, int* g) {
  const int lane = (int)(threadIdx.x & 31u);
  const unsigned int* flag = nullptr;
  unsigned int target = 0;
  if (lane < 9) {
    const int ty = (int)fdiv((uint32_t)t, G.div_x), tx = t - ty * G.tiles_x;
    int ny = ty + lane / 3 - 1, nx = tx + lane % 3 - 1;  // periodic neighbours
    ny = (ny < 0) ? ny + G.tiles_y : (ny >= G.tiles_y ? ny - G.tiles_y : ny);
    nx = (nx < 0) ? nx + G.tiles_x : (nx >= G.tiles_x ? nx - G.tiles_x : nx);
    flag = &prog[ny * G.tiles_x + nx];
    target = (unsigned int)r;
  } else if (lane == 9) {
    flag = &H->vring[r % kWaveRing].tag;
    target = (unsigned int)(r + 1);
  } else if (lane == 10 && r >= kWaveRing) {
    flag = &H->committed;
    target = (unsigned int)(r - kWaveRing + 1);
  }
  unsigned int used = 0;
  bool ok;
  for (;;) {
    const bool mine = (flag == nullptr) || ld_acquire(flag) >= target;
    ok = __all_sync(0xFFFFFFFFu, mine);
    if (ok || !block) break;
    const bool stop = *(volatile unsigned int*)&H->abort != 0u;
    if (__any_sync(0xFFFFFFFFu, stop)) return false;
    if (++used > kWaitPollLimit) {
      if (lane == 0) {
        atomicOr(err, 1u);
        atomicExch(&H->abort, 1u);
      }
      return false;
    }
    __nanosleep(128);
  }
  // lane 9 acquired the move: its gate reaches the other lanes by shuffle
  int gv = 0;
  if (lane == 9) gv = *(volatile int*)&H->vring[r % kWaveRing].g;
  *g = __shfl_sync(0xFFFFFFFFu, gv, 9);
  return ok;
}

// Publishes the move of relative step r in its ring slot.
__device__ __forceinline__ void wave_publish(WaveHdr* H, long long r, const VolumeResult& m) {
  WaveMove& w = H->vring[r % kWaveRing];
  volatile WaveMove* vw = &w;
  vw->V = m.V;
  vw->u = m.u;
  vw->g = m.g;
  vw->acc = m.accepted;
  st_release_u32(&w.tag, (unsigned int)(r + 1));
}

// Commit of relative step r (one thread; the previous step is committed):
// finalize_step's bookkeeping with the counts from the step's slot and the
// step's move from the ring.
__device__ void wave_commit(const LatticeArgs& A, WaveHdr* H, long long step0, long long r) {
  volatile Ctrl* c = A.ctrl;
  volatile WaveAcc* a = &H->acc[r % kWaveRing];
  volatile WaveMove* m = &H->vring[r % kWaveRing];
  const int every = c->record_every;
  const long long sweep = step0 + r;
  Ctrl s;
  const bool recorded = (every > 0) && ((sweep + 1) % every == 0);
  s.n_hb_raw = c->n_hb_raw + (long long)a->hb;
  s.n_coop = c->n_coop + (long long)a->pairs;
  s.acc_sigma = c->acc_sigma + (long long)a->moves;
  s.V_iso = m->V;
  s.u_cell = m->u;
  s.g = m->g;
  s.acc_volume = c->acc_volume + m->acc;
  s.sweep = sweep + 1;
  c->n_hb_raw = s.n_hb_raw;
  c->n_coop = s.n_coop;
  c->acc_sigma = s.acc_sigma;
  c->V_iso = s.V_iso;
  c->u_cell = s.u_cell;
  c->g = s.g;
  c->acc_volume = s.acc_volume;
  c->sweep = s.sweep;
  if (recorded) {
    const long long head = c->ring_head;
    s.error = c->error;
    for (int v = 0; v < 8; ++v) {
      s.hist[v] = (long long)a->hist[v];
      c->hist[v] = s.hist[v];
    }
    A.ring[head % A.ring_cap] = make_obs(*A.vol, &s);
    c->ring_head = head + 1;
  }
  a->hb = 0;
  a->pairs = 0;
  a->moves = 0;
  for (int v = 0; v < 8; ++v) a->hist[v] = 0;
  a->done = 0;
  st_release_u32(&H->committed, (unsigned int)(r + 1));
}

// WALK: every tile full and the rows 16-byte aligned (the column-walking
// colour phases; a separate instantiation, as for k_sweep_tiled).
template <int RNG_WORDS, bool CMP64, int TR, int TW, bool WALK>
__global__ void __launch_bounds__(kThreads, kWaveBlocksPerSM)
    k_sweep_wave(const __grid_constant__ LatticeArgs A, WaveHdr* H, long long step0,
                 long long n_steps, const __grid_constant__ WaveGeom G,
                 const __grid_constant__ CUtensorMap tm0, const __grid_constant__ CUtensorMap tm1) {
  __shared__ union {
    TileSmem<TR, TW> tile;
    VolumeArgs vol;  // the engine block's copy of the parameters
  } U;
  __shared__ Tables2 Tb;
  __shared__ uint32_t s_hist4[4];
  // s_staged: 0 the item is not staged, 1 staged by cp.async, 2 by TMA
  __shared__ int s_r, s_t, s_ok, s_g, s_staged, n_r, n_t, n_ok, n_ready, n_g;
  __shared__ alignas(8) uint64_t s_bar;
  Ctrl* const ctl = A.ctrl;
  unsigned int* const err = &ctl->error;

  if (blockIdx.x == 0) {
    // The engine: the volume move of every step of the call, and of the
    // first step of the next one, each from the move before it.
    __shared__ double s_xch;
    __shared__ VolumeResult s_res;
    __shared__ int s_go;
    VolumeArgs* sV = &U.vol;
    stage_volume_args(sV, A.vol);
    __syncthreads();
    if (threadIdx.x >= 64) return;
    const int role = (int)(threadIdx.x >> 5);
    volatile Ctrl* c = ctl;
    VolumeResult cur;
    cur.V = c->next_V;
    cur.u = c->next_u;
    cur.g = c->next_g;
    cur.accepted = c->next_acc;
    if (threadIdx.x == 0) wave_publish(H, 0, cur);
    bool alive = true;
    for (long long r = 1; r <= n_steps; ++r) {
      if (threadIdx.x == 0)
        s_go = (r < kWaveRing) ? 1
                               : (wave_wait_geq(&H->committed, (unsigned int)(r - kWaveRing + 1), H,
                                                err) ? 1 : 0);
      engine_sync();
      if (!s_go) {
        alive = false;
        break;
      }
      VolumeResult res;
      const bool ok = volume_decide_pair<3>(role, *sV, step0 + r, cur.V, cur.u, cur.g, -1,
                                            A.keys, &res, &s_xch);
      if (!ok) {
        // the proposal changes the gate: decide it with the bonds after step r - 1
        if (threadIdx.x == 0) s_go = wave_wait_geq(&H->committed, (unsigned int)r, H, err) ? 1 : 0;
        engine_sync();
        if (!s_go) {
          alive = false;
          break;
        }
        const long long nhb = c->n_hb_raw;
        volume_decide_pair<3>(role, *sV, step0 + r, cur.V, cur.u, cur.g, nhb, A.keys, &res,
                              &s_xch);
      }
      if (threadIdx.x == 0) s_res = res;  // valid in role 0's lanes
      engine_sync();
      cur = s_res;
      engine_sync();  // every thread has read s_res before the next write
      if (r < n_steps && threadIdx.x == 0) wave_publish(H, r, cur);
    }
    if (alive && threadIdx.x == 0) {
      c->next_V = cur.V;
      c->next_u = cur.u;
      c->next_g = cur.g;
      c->next_acc = cur.accepted;
      c->ahead_state = 0;
    }
    return;
  }

  TileSmem<TR, TW>& S = U.tile;
  const int L = A.L, Lh = L >> 1;
  const long long N = (long long)L * L;
  const int T = G.T;
  const long long total = n_steps * (long long)T;
  unsigned int* const prog = reinterpret_cast<unsigned int*>(H + 1);
  const int every = ctl->record_every;
  const bool async16 = (L % 8) == 0;  // rows and tile origins on 16-byte boundaries
  fill_prop2(Tb, A.q);
  if (threadIdx.x < 4) s_hist4[threadIdx.x] = 0;
  if (threadIdx.x == 0) mbar_init(&s_bar, 1);  // before the loop's first barrier
  uint32_t parity = 0;
  int g_cur = -1;
  TileCounts cnt{0, 0, 0};  // this thread's counts of the tiles not yet reported
  int pend = 0;             // the block's tiles not yet reported (all of one step)

  // take an item and, blocking, wait for it (warp 0)
  if (threadIdx.x < 32) {
    unsigned long long i = 0;
    if (threadIdx.x == 0) i = atomicAdd(&H->next, 1ull);
    i = __shfl_sync(0xFFFFFFFFu, i, 0);
    const bool have = (long long)i < total;
    int g = 0, r = 0, t = 0;
    if (have) wave_item(G, i, &r, &t);
    const bool ok = have && wave_deps(H, prog, r, t, G, true, err, &g);
    if (threadIdx.x == 0) {
      s_ok = ok ? 1 : 0;
      s_r = r;
      s_t = t;
      s_g = g;
      s_staged = 0;
    }
  }
  for (;;) {
    __syncthreads();
    if (!s_ok) break;
    const int r = s_r, t = s_t, g = s_g, staged = s_staged;
    const long long step = step0 + r;
    if (g != g_cur) {  // block-uniform
      fill_rows2(Tb, A.table24, g);
      g_cur = g;
    }
    StepView<KeysStep> v;
    v.src = reinterpret_cast<const uint32_t*>(A.state + (size_t)(step & 1) * N);
    v.dst = reinterpret_cast<uint32_t*>(A.state + (size_t)((step + 1) & 1) * N);
    v.L = L;
    v.Lh = Lh;
    v.q = A.q;
    v.s_lo = (uint32_t)((unsigned long long)step & 0xFFFFFFFFu);
    v.s_hi = (uint32_t)((unsigned long long)step >> 32);
    v.keys.K = A.keys;
    v.keys.sd = step_draw(v.s_lo, v.s_hi, A.keys);
    v.err = err;
    const int ty = (int)fdiv((uint32_t)t, G.div_x);
    const TileGeom gm = tile_geom<TR, TW>(L, Lh, ty * TR, (t - ty * G.tiles_x) * TW);
    if (!staged) {
      // the words were written by other SMs during this launch: through L2
      if (async16)
        stage_async16<TR, TW, kThreads>(v, gm, S);
      else
        stage_plain<TR, TW, kThreads, true>(v, gm, S);
    }
    if (staged == 2) {  // block-uniform: the TMA copy started during the last item
      uint32_t spins = 0;
      while (!mbar_try_wait(&s_bar, parity)) {
        if (++spins > kWaveTmaWaitLimit) {  // a copy that never lands: stop the launch
          atomicOr(err, 1u);
          atomicExch(&H->abort, 1u);
          break;
        }
      }
      parity ^= 1u;
    } else {
      cp_async_wait_all();
    }
    __syncthreads();
    const bool rec = step_recorded(every, step);
    if constexpr (WALK) {
      if (rec)
        colour0_walk<RNG_WORDS, CMP64, TR, TW, kThreads, true, 2>(v, gm, S, Tb, cnt, s_hist4);
      else
        colour0_walk<RNG_WORDS, CMP64, TR, TW, kThreads, false, 2>(v, gm, S, Tb, cnt, nullptr);
    } else {
      colour0<RNG_WORDS, CMP64, TR, TW, kThreads, kWaveShape>(v, gm, S, Tb, cnt,
                                                               rec ? s_hist4 : nullptr);
    }
    // S.in is free: the last warp (the least colour-0 work) takes the next
    // item and, when its dependencies already hold, it is staged while
    // colour 1 runs
    if ((int)(threadIdx.x >> 5) == kThreads / 32 - 1) {
      unsigned long long i = 0;
      if ((threadIdx.x & 31u) == 0) i = atomicAdd(&H->next, 1ull);
      i = __shfl_sync(0xFFFFFFFFu, i, 0);
      const bool have = (long long)i < total;
      int g2 = 0, r2 = 0, t2 = 0;
      if (have) wave_item(G, i, &r2, &t2);
      const bool ready = have && wave_deps(H, prog, r2, t2, G, false, err, &g2);
      if ((threadIdx.x & 31u) == 0) {
        n_ok = have ? 1 : 0;
        n_r = r2;
        n_t = t2;
        n_g = g2;
        n_ready = (ready && async16) ? 1 : 0;
      }
    }
    __syncthreads();
    bool next_tma = false;
    if (n_ready) {
      StepView<KeysInRegs> vn;
      vn.src = reinterpret_cast<const uint32_t*>(A.state + (size_t)((step0 + n_r) & 1) * N);
      vn.L = L;
      vn.Lh = Lh;
      vn.err = err;
      const int nty = (int)fdiv((uint32_t)n_t, G.div_x);
      const TileGeom gn = tile_geom<TR, TW>(L, Lh, nty * TR, (n_t - nty * G.tiles_x) * TW);
      // 64 x 64-word tiles: one TMA box (issued by thread 0) when the tile
      // and its halo lie inside the lattice (the box's x, p0 - 4, is a
      // multiple of 4 words); at 4096^2 106.7 against 108.6 us per step with
      // cp.async.  The smaller tiles keep the 16-byte cp.async copies, which
      // ran 1-2 % faster there (1024^2 with 16 x 32 words: 11.2 against
      // 11.4 us; 2048^2 with 32 x 32: 32.8 against 33.3).
      next_tma = TR >= 64 && A.use_tma && gn.th == TR && gn.tw == TW && gn.p0 >= 4 &&
                 gn.p0 + TW + 4 <= Lh && gn.y0 >= 2 && gn.y0 + TR + 2 <= L;
      if (next_tma) {
        if (threadIdx.x == 0) {
          // S.in's colour-0 reads are done (the barrier above); the words
          // of the tiles around were acquired by the dependency test (warp
          // NT/32 - 1, before the barrier) and are read by the async proxy
          fence_proxy_async_shared();
          fence_proxy_async_global();
          if (dcheck(((gn.p0 - 4) & 3) == 0 && gn.y0 - 2 >= 0 && gn.p0 + TW + 4 <= Lh &&
                         gn.y0 + TR + 2 <= L,
                     err, kSiteTma)) {
            mbar_arrive_expect_tx(&s_bar, (uint32_t)sizeof(S.in));
            tma_load_2d(&S.in[0][0], ((step0 + n_r) & 1) ? &tm1 : &tm0, gn.p0 - 4, gn.y0 - 2,
                        &s_bar);
          } else {
            mbar_arrive_expect_tx(&s_bar, 0u);
          }
        }
      } else {
        stage_async16<TR, TW, kThreads>(vn, gn, S);
      }
    }
    if constexpr (WALK) {
      if (rec)
        colour1_walk<RNG_WORDS, CMP64, TR, TW, kThreads, true, 2>(v, gm, S, Tb, cnt, s_hist4);
      else
        colour1_walk<RNG_WORDS, CMP64, TR, TW, kThreads, false, 2>(v, gm, S, Tb, cnt, nullptr);
    } else {
      colour1<RNG_WORDS, CMP64, TR, TW, kThreads, kWaveShape>(v, gm, S, Tb, cnt,
                                                               rec ? s_hist4 : nullptr);
    }
    WaveAcc* slot = &H->acc[r % kWaveRing];
    if (rec) {  // block-uniform
      __syncthreads();
      hist_flush(s_hist4, slot->hist);
    }
    __syncthreads();  // the tile's stores (and N_q' adds) are done
    if (threadIdx.x == 0) {
      // the tile's words to the tiles of the next step around it: a fence
      // (releasing what the block's barrier ordered) and a relaxed store
      fence_acq_rel_gpu();
      st_relaxed_u32(&prog[t], (unsigned int)(r + 1));
    }
    ++pend;
    // The counts of consecutive tiles of one step stay in the threads'
    // registers and are reported together when the block's next item is of
    // another step, is not ready (the block is about to wait: nothing it
    // holds may be what others wait for) or does not exist.
    if (!n_ok || !n_ready || n_r != r) {  // block-uniform
      uint32_t dhb = (uint32_t)cnt.dhb(), dc = (uint32_t)cnt.dc(), nacc = cnt.nacc;
      block_sum3<kThreads>(dhb, dc, nacc);
      if (threadIdx.x == 0) {
        atomicAdd(&slot->hb, (unsigned long long)(long long)(int)dhb);
        atomicAdd(&slot->pairs, (unsigned long long)(long long)(int)dc);
        atomicAdd(&slot->moves, (unsigned long long)nacc);
        // the counts before the completion count; the tile that completes
        // the step commits it after the step before (its fence acquires
        // every other tile's counts, released the same way)
        fence_acq_rel_gpu();
        if (atom_add_relaxed_u32(&slot->done, (unsigned int)pend) + (unsigned int)pend ==
            (unsigned int)T) {
          fence_acq_rel_gpu();
          if (r == 0 || wave_wait_geq(&H->committed, (unsigned int)r, H, err))
            wave_commit(A, H, step0, r);
        }
      }
      cnt = TileCounts{0, 0, 0};
      pend = 0;
    }
    // the next item becomes the current one; if it could not be staged yet,
    // warp 0 waits for it
    if (threadIdx.x < 32) {
      const bool have = n_ok != 0;
      bool ok = have;
      int g2 = n_g;
      if (have && !n_ready) ok = wave_deps(H, prog, n_r, n_t, G, true, err, &g2);
      if (threadIdx.x == 0) {
        s_ok = ok ? 1 : 0;
        s_r = n_r;
        s_t = n_t;
        s_g = g2;
        s_staged = n_ready ? (next_tma ? 2 : 1) : 0;
      }
    }
  }
  cp_async_wait_all();  // no copy may still be in flight when the block exits
}

template <int RW, bool C64, int TR, int TW>
const void* wave_kernel_s(int L) {
  const bool walk = L % TR == 0 && (L / 2) % TW == 0 && (L / 2) % 4 == 0;
  return walk ? (const void*)k_sweep_wave<RW, C64, TR, TW, true>
              : (const void*)k_sweep_wave<RW, C64, TR, TW, false>;
}

template <int RW, bool C64>
const void* wave_kernel_t(int shape, int L) {
  switch (shape) {
    case 0: return wave_kernel_s<RW, C64, 64, 64>(L);
    case 1: return wave_kernel_s<RW, C64, 32, 32>(L);
    default: return wave_kernel_s<RW, C64, 16, 32>(L);
  }
}

// The kernel for (rng_words, cmp64, tile shape, lattice side); L = 1 names
// the general form (both forms have the same registers and shared memory).
const void* wave_kernel(int rng_words, bool cmp64, int shape, int L) {
  if (rng_words == 1)
    return cmp64 ? wave_kernel_t<1, true>(shape, L) : wave_kernel_t<1, false>(shape, L);
  return cmp64 ? wave_kernel_t<2, true>(shape, L) : wave_kernel_t<2, false>(shape, L);
}

}  // namespace

int wave_blocks(int rng_words, bool cmp64, int shape) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wave_kernel(rng_words, cmp64, shape, 1),
                                                    kThreads, 0) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * sm_count();
}

cudaError_t launch_wave(const LatticeArgs& A, WaveHdr* H, size_t scratch_bytes, int rng_words,
                        bool cmp64, int shape, long long step0, long long n_steps,
                        const CUtensorMap* tm, cudaStream_t s) {
  const int grid = wave_blocks(rng_words, cmp64, shape);
  if (grid < 2) return cudaErrorCooperativeLaunchTooLarge;
  const int tr = (shape == 0) ? 64 : (shape == 1) ? 32 : 16, tw = (shape == 0) ? 64 : 32;
  WaveGeom G;
  G.tiles_x = (A.L / 2 + tw - 1) / tw;
  G.tiles_y = (A.L + tr - 1) / tr;
  G.T = G.tiles_x * G.tiles_y;
  G.div_T = make_fastdiv((uint32_t)G.T);
  G.div_x = make_fastdiv((uint32_t)G.tiles_x);
  G.small = (n_steps * (long long)G.T < (1ll << 31)) ? 1 : 0;
  cudaError_t e = cudaMemsetAsync(H, 0, scratch_bytes, s);
  if (e != cudaSuccess) return e;
  void* args[7] = {const_cast<LatticeArgs*>(&A), &H, &step0, &n_steps, &G,
                   const_cast<CUtensorMap*>(&tm[0]), const_cast<CUtensorMap*>(&tm[1])};
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, wave_kernel(rng_words, cmp64, shape, (int)A.L), args);
}

}  // namespace cvf
