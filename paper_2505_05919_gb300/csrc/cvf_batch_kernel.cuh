// cvf_batch_kernel.cuh -- the persistent batched sweep (device side), shared
// by the translation units that instantiate it for each block size.
//
// Work items are (relative step s, replica r, tile t), dequeued from one
// atomic counter in step-major order.  An item waits until replica r has
// completed s steps in this launch (a bounded spin on a per-replica progress
// counter, acquire/release); the last tile of a replica-step commits the step
// (counts, volume move, observables: finalize_step) and releases the
// replica's next step.  Items are processed one at a time in dequeue order by
// co-resident blocks, so the oldest unfinished item can always run: there is
// no deadlock, and a wait that still exceeds its limit sets an error word and
// ends the launch (reported as CVF_ETIMEOUT).  Every replica computes exactly
// what it computes alone (same tile code, same counter-based draws).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "cvf.h"
#include "cvf_device.cuh"
#include "cvf_lattice.cuh"
#include "cvf_tile.cuh"

namespace cvf {

struct ReplicaDesc {
  uint16_t* state;  // state pair, 2 * L * L words
  Ctrl* ctrl;
  const unsigned long long* table24;
  const VolumeArgs* vol;
  cvf_obs* ring;
  long long ring_cap;
  RoundKeys keys;
  int32_t L;
  uint32_t q;
};

// colour loops: the single-lattice sweep's shape (over the 256 mixed-size
// replicas: 497 sigma-updates/ns; 487 with two cells per iteration in both
// colours and the half a runtime value, 481 with that and the recorded-step
// copy, 472 with one loop per half and one cell per iteration)
constexpr int kBatchShape = kHalfRows | kUnroll1 | kSplitRec;

// Launch description written by the host before every launch.
constexpr int kBatchMaxSegments = 64;
struct BatchWork {
  unsigned long long next;   // item counter
  unsigned long long pad_next[15];  // the counter alone in its 128-byte line: every
                                    // claim is an atomic on it, every wait reads `error`
  unsigned int error;        // 1: a wait gave up; 0x100 + site: a debug index check failed
  unsigned int pad;
  long long total_items;
  int32_t n_active;          // replicas advanced by this launch
  int32_t nseg;
  int32_t tile_rows, tile_words;
  long long seg_s0[kBatchMaxSegments + 1];    // first relative step of each segment
  long long seg_base[kBatchMaxSegments + 1];  // first item of each segment
  int32_t seg_active[kBatchMaxSegments];      // active replicas (prefix of `order`)
  // followed in device memory by: int32 order[n_active], int64 tile_prefix[n_active + 1],
  // uint32 progress[n_replicas]
};


__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Takes the next work item from the launch's counter and decodes it.  Called
// by all 32 lanes of one warp; every lane returns the same value, the item is
// valid in lane 0.  The replica of the item is found by a 32-way search of
// the strictly increasing tile_prefix (two rounds of parallel loads for up to
// 1024 replicas, where a binary search takes a dependent load per halving);
// false when the launch is out of items or has failed.
__device__ __forceinline__ bool take_item(BatchWork* W, const int32_t* __restrict__ order,
                                          const long long* __restrict__ tile_prefix, int* rep,
                                          int* tile, long long* rel) {
  const unsigned int lane = threadIdx.x & 31u;
  unsigned long long i = 0;
  int stop = 0;
  if (lane == 0u) {
    i = atomicAdd(&W->next, 1ull);
    stop = ((long long)i >= W->total_items || *(volatile unsigned int*)&W->error) ? 1 : 0;
  }
  i = __shfl_sync(0xFFFFFFFFu, i, 0);
  if (__shfl_sync(0xFFFFFFFFu, stop, 0)) return false;
  // segment, relative step, replica, tile
  int k = 0;
  while (k + 1 < W->nseg && (long long)i >= W->seg_base[k + 1]) ++k;
  const int A = W->seg_active[k];
  const long long T = tile_prefix[A];
  const long long r = (long long)i - W->seg_base[k];
  const long long s = W->seg_s0[k] + r / T;
  const long long j = r % T;
  int lo = 0, hi = A;  // largest ri with tile_prefix[ri] <= j
  while (hi - lo > 1) {
    const int span = (hi - lo + 31) / 32;
    const int idx = lo + (int)lane * span;
    const bool in = idx < hi && tile_prefix[idx] <= j;
    const unsigned int m = __ballot_sync(0xFFFFFFFFu, in);  // bit 0 always set
    lo += (31 - __clz((int)m)) * span;
    hi = min(hi, lo + span);
  }
  int ok = 1;
  if (lane == 0u) {
    ok = dcheck(k < W->nseg && A <= W->n_active && lo >= 0 && lo < A && j >= 0 && j < T &&
                    j < tile_prefix[lo + 1] && s >= 0,
                &W->error, kSiteBatchItem) ? 1 : 0;
    *rep = order[lo];
    *tile = (int)(j - tile_prefix[lo]);
    *rel = s;
  }
  return __shfl_sync(0xFFFFFFFFu, ok, 0) != 0;
}

// The persistent batched sweep.  A block works through items (step s,
// replica r, tile t) in counter order.  After an item's first colour, when
// the S.in buffer is free, it takes its next item; if that item's replica
// has already finished the steps before it, the next tile's rows are copied
// in (16-byte cp.async through L2, lattices with L a multiple of 8) while the
// second colour runs.  Otherwise the item waits (bounded) and stages its tile
// when it comes up.  A block only waits for items taken before its own, so
// the oldest unfinished item can always run.
// Blocks per SM the register budget is sized for: 5 x 256 threads, 10 x 128;
// 512-thread blocks get 2 (64 registers a thread instead of 48).
constexpr int batch_min_blocks(int nt) { return nt >= 512 ? 2 : kBatchBlocksPerSM * kThreads / nt; }

template <int RNG_WORDS, bool CMP64, int TR, int TW, int NT>
__global__ void __launch_bounds__(NT, batch_min_blocks(NT))
    k_batch_sweep(const ReplicaDesc* __restrict__ reps, BatchWork* W,
                  const int32_t* __restrict__ order, const long long* __restrict__ tile_prefix,
                  unsigned int* progress) {
  __shared__ TileSmem<TR, TW> S;
  __shared__ Tables2 Tb;
  __shared__ int s_rep, s_tile, s_valid, s_staged, s_abort, s_last;
  __shared__ long long s_rel;
  __shared__ int n_rep, n_tile, n_valid, n_ready;
  __shared__ long long n_rel;
  __shared__ uint32_t s_q;
  __shared__ uint32_t s_hist4[4];
  __shared__ RoundKeys s_keys;  // the current replica's round keys (copied into registers per item)
  __shared__ double s_xch;      // the volume item's two warps' exchange
  __shared__ int s_tab_rep, s_tab_g, s_key_rep;  // whose rows / keys Tb and s_keys hold
  // a replica's step count when the launch began (s_step_rep's): only this
  // launch advances it, so an item of relative step rel runs at step
  // s_step0 + rel once the replica's progress reached rel
  __shared__ int s_step_rep;
  __shared__ long long s_step0;
  if (threadIdx.x == 0) {
    s_tab_rep = -1;
    s_tab_g = -1;
    s_key_rep = -1;
    s_step_rep = -1;
  }
  if (threadIdx.x < 32) {
    int r = 0, t = 0;
    long long e = 0;
    const bool ok = take_item(W, order, tile_prefix, &r, &t, &e);
    if (threadIdx.x == 0) {
      s_q = 0;
      s_valid = ok ? 1 : 0;
      s_rep = r;
      s_tile = t;
      s_rel = e;
      s_staged = 0;
    }
  }
  if (threadIdx.x < 4) s_hist4[threadIdx.x] = 0;
  for (;;) {
    __syncthreads();
    if (!s_valid) break;
    if (threadIdx.x == 0) {
      int abort = 0;
      if (!s_staged) {
        // wait until the replica has completed the item's earlier steps
        const WaitResult wr = wait_flag_geq(&progress[s_rep], (unsigned int)s_rel, &W->error,
                                            kWaitPollLimit);
        if (wr != kWaitDone) {
          if (wr == kWaitGaveUp) atomicExch(&W->error, 1u);
          abort = 1;
        }
      }
      s_abort = abort;
    }
    __syncthreads();
    if (s_abort) break;
    const int rep = s_rep, t = s_tile, staged = s_staged;
    const long long rel = s_rel;
    const ReplicaDesc& R = reps[rep];
    Ctrl* ctl = R.ctrl;
    volatile Ctrl* vc = ctl;
    const long long step = (rep == s_step_rep) ? s_step0 + rel : vc->sweep;
    const int tiles_x = (R.L / 2 + TW - 1) / TW;
    const int ntiles = tiles_x * ((R.L + TR - 1) / TR);
    if (t == ntiles) {
      // The volume item: the move of the replica's next step, decided while
      // the step's tiles run (it does not depend on the bonds unless the gate
      // would flip; then the step's commit decides it with the new bonds).
      if (threadIdx.x < 64) {  // warps 0 and 1: the move on two FP64 pipes
        VolumeResult r;
        const bool ok = volume_decide_pair<3>((int)(threadIdx.x >> 5), *R.vol, step + 1,
                                              vc->next_V, vc->next_u, vc->next_g, -1, R.keys, &r,
                                              &s_xch);
        if (threadIdx.x == 0 && ok) {
          vc->ahead_V = r.V;
          vc->ahead_u = r.u;
          vc->ahead_g = r.g;
          vc->ahead_acc = r.accepted;
          vc->ahead_state = 1;
        }
      }
      if (threadIdx.x == 0) {
        // release: the decision is visible to the step's committer; acquire:
        // the committer sees every item's counts
        if (atom_add_acq_rel(&ctl->done, 1u) == (unsigned int)ntiles) {
          finalize_step<true>(*R.vol, ctl, R.ring, R.ring_cap, R.keys);
          st_release(&progress[rep], (unsigned int)(rel + 1));
        }
      }
      // the last warp takes the next item while warps 0 and 1 decide
      if ((int)(threadIdx.x >> 5) == NT / 32 - 1) {
        int rr = 0, tt = 0;
        long long e = 0;
        const bool ok = take_item(W, order, tile_prefix, &rr, &tt, &e);
        if ((threadIdx.x & 31) == 0) {
          s_valid = ok ? 1 : 0;
          s_rep = rr;
          s_tile = tt;
          s_rel = e;
          s_staged = 0;
        }
      }
      continue;
    }
    // the gate of a step is fixed once its items can run, so every thread
    // reads the same g; its load is in flight while the tile is staged
    const int g = vc->next_g;
    if (s_q != R.q) {  // block-uniform
      fill_prop2(Tb, R.q);
      __syncthreads();
      if (threadIdx.x == 0) s_q = R.q;
    }
    const int L = R.L, Lh = L >> 1;
    const long long N = (long long)L * L;
    using Keys = KeysStep;
    StepView<Keys> v;
    v.src = reinterpret_cast<const uint32_t*>(R.state + (size_t)(step & 1) * N);
    v.dst = reinterpret_cast<uint32_t*>(R.state + (size_t)((step + 1) & 1) * N);
    v.L = L;
    v.Lh = Lh;
    v.q = R.q;
    v.s_lo = (uint32_t)((unsigned long long)step & 0xFFFFFFFFu);
    v.s_hi = (uint32_t)((unsigned long long)step >> 32);
    v.err = &W->error;
    const TileGeom gm = tile_geom<TR, TW>(L, Lh, (t / tiles_x) * TR, (t % tiles_x) * TW);
    if (staged)
      cp_async_wait_all();
    else
      stage_plain<TR, TW, NT, true>(v, gm, S);
    // the threshold rows and round keys stay from the block's previous item
    // when it had the same replica (and gate)
    if (rep != s_tab_rep || g != s_tab_g) fill_rows2(Tb, R.table24, g);
    if (rep != s_key_rep && threadIdx.x < 10) {
      s_keys.k[threadIdx.x] = R.keys.k[threadIdx.x];
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // read again only after a later barrier
      s_tab_rep = rep;
      s_tab_g = g;
      s_key_rep = rep;
      s_step_rep = rep;
      s_step0 = step - rel;
    }
    // the replica's keys by value and the step's folded first Philox rounds
    // (KeysStep; the batched workload on 64 x 64-word tiles: 126.6 -> 125.7
    // us per step, on 32 x 32: 137.8 -> 134.4, against the keys read from
    // shared memory in every round), after the barrier above
    v.keys.K = s_keys;
    v.keys.sd = step_draw(v.s_lo, v.s_hi, s_keys);
    TileCounts cnt{0, 0, 0};
    const bool rec = step_recorded(vc->record_every, step);
    // replicas whose tiles are all full (and rows 16-byte aligned) take the
    // column-walking colour phases where the block shape allows them (each
    // thread group an even number of rows): the 256 replicas of the batched
    // workload on 64 x 64-word tiles, 140.8 -> 126.4 us per step
    constexpr bool kWalkShape =
        NT % TW == 0 && TR % (NT / TW) == 0 && (TR / (NT / TW)) % 2 == 0;
    const bool walk = kWalkShape && L % TR == 0 && Lh % TW == 0 && (Lh & 3) == 0;
    if constexpr (kWalkShape) {
      if (walk) {
        if (rec)
          colour0_walk<RNG_WORDS, CMP64, TR, TW, NT, true, 1>(v, gm, S, Tb, cnt, s_hist4);
        else
          colour0_walk<RNG_WORDS, CMP64, TR, TW, NT, false, 1>(v, gm, S, Tb, cnt, nullptr);
      }
    }
    if (!walk)
      colour0<RNG_WORDS, CMP64, TR, TW, NT, kBatchShape>(v, gm, S, Tb, cnt, rec ? s_hist4 : nullptr);
    // S.in is free: take the next item and, when it can start, copy its tile.
    // The last warp takes it: it has the fewest rows (and no ring cells) in
    // the first colour, so the take overlaps the other warps' remaining work.
    if ((int)(threadIdx.x >> 5) == NT / 32 - 1) {
      int r = 0, tt = 0;
      long long e = 0;
      const bool ok = take_item(W, order, tile_prefix, &r, &tt, &e);
      if ((threadIdx.x & 31) == 0) {
        n_valid = ok ? 1 : 0;
        n_rep = r;
        n_tile = tt;
        n_rel = e;
        const int nl = reps[r].L;
        const int ntn = ((nl / 2 + TW - 1) / TW) * ((nl + TR - 1) / TR);
        n_ready = (n_valid && tt < ntn && nl % 8 == 0 &&
                   ld_acquire(&progress[r]) >= (unsigned int)e) ? 1 : 0;
      }
    }
    __syncthreads();
    if (n_ready) {
      const ReplicaDesc& Rn = reps[n_rep];
      const int Ln = Rn.L, Lhn = Ln >> 1;
      const long long Nn = (long long)Ln * Ln;
      const long long step_n =
          (n_rep == s_step_rep) ? s_step0 + n_rel : ((volatile Ctrl*)Rn.ctrl)->sweep;
      StepView<KeysRound> vn;
      vn.src = reinterpret_cast<const uint32_t*>(Rn.state + (size_t)(step_n & 1) * Nn);
      vn.L = Ln;
      vn.Lh = Lhn;
      vn.err = &W->error;
      const int tx = (Lhn + TW - 1) / TW;
      const TileGeom gn = tile_geom<TR, TW>(Ln, Lhn, (n_tile / tx) * TR, (n_tile % tx) * TW);
      stage_async16<TR, TW, NT>(vn, gn, S);
    }
    if constexpr (kWalkShape) {
      if (walk) {
        if (rec)
          colour1_walk<RNG_WORDS, CMP64, TR, TW, NT, true, 1>(v, gm, S, Tb, cnt, s_hist4);
        else
          colour1_walk<RNG_WORDS, CMP64, TR, TW, NT, false, 1>(v, gm, S, Tb, cnt, nullptr);
      }
    }
    if (!walk)
      colour1<RNG_WORDS, CMP64, TR, TW, NT, kBatchShape>(v, gm, S, Tb, cnt, rec ? s_hist4 : nullptr);
    if (rec) {  // block-uniform: only on recorded steps
      __syncthreads();
      hist_flush(s_hist4, ctl->acc_hist);
    }
    uint32_t dhb = (uint32_t)cnt.dhb(), dc = (uint32_t)cnt.dc(), nacc = cnt.nacc;
    block_sum3<NT>(dhb, dc, nacc);  // two's complement sums
    if (threadIdx.x == 0) {
      atomicAdd(&ctl->acc_hb, (unsigned long long)(long long)(int)dhb);
      atomicAdd(&ctl->acc_pairs, (unsigned long long)(long long)(int)dc);
      atomicAdd(&ctl->acc_moves, (unsigned long long)nacc);
      // after the block's barrier: releases the tile's words and counts to the
      // step's committer (ntiles tiles + the volume item), which acquires them
      s_last = (atom_add_acq_rel(&ctl->done, 1u) == (unsigned int)ntiles) ? 1 : 0;
      if (s_last) {
        finalize_step<true>(*R.vol, ctl, R.ring, R.ring_cap, R.keys);
        st_release(&progress[rep], (unsigned int)(rel + 1));
      }
      // the next item becomes the current one
      s_valid = n_valid;
      s_rep = n_rep;
      s_tile = n_tile;
      s_rel = n_rel;
      s_staged = n_ready;
    }
  }
  cp_async_wait_all();  // no copy may still be in flight when the block exits
}

}  // namespace cvf

namespace cvf {

// The kernel of one (RNG words, 64-bit thresholds, tile rows x words, block
// threads) combination, as a launchable pointer.
using BatchKernelFn = void (*)(const ReplicaDesc*, BatchWork*, const int32_t*, const long long*,
                               unsigned int*);

template <int NT>
BatchKernelFn batch_kernel_for(int rng_words, bool cmp64, int shape) {
  auto pick = [&](auto rw, auto c64) -> BatchKernelFn {
    constexpr int RW = decltype(rw)::value;
    constexpr bool C64 = decltype(c64)::value;
    switch (shape) {
      case 0: return k_batch_sweep<RW, C64, 64, 64, NT>;
      case 1: return k_batch_sweep<RW, C64, 32, 32, NT>;
      case 2: return k_batch_sweep<RW, C64, 32, 16, NT>;
      default: return k_batch_sweep<RW, C64, 16, 16, NT>;
    }
  };
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;
  if (rng_words == 1)
    return cmp64 ? pick(I1{}, std::true_type{}) : pick(I1{}, std::false_type{});
  return cmp64 ? pick(I2{}, std::true_type{}) : pick(I2{}, std::false_type{});
}

// Defined in cvf_batch_nt128.cu / cvf_batch_nt512.cu: the kernels with
// 128- and 512-thread blocks.
BatchKernelFn batch_kernel_nt128(int rng_words, bool cmp64, int shape);
BatchKernelFn batch_kernel_nt512(int rng_words, bool cmp64, int shape);

}  // namespace cvf
