// cvf_batch.cu -- many independent lattices ("replicas": differing L, q, T,
// P, seeds) advanced by one persistent, cooperative, graph-captured launch.
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
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "cvf.h"
#include "cvf_device.cuh"
#include "cvf_host.h"
#include "cvf_lattice.cuh"
#include "cvf_tile.cuh"

using namespace cvf;

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

// A replica's tables from the call's parameters (passed by value, so the
// caller's host memory is free as soon as the launch is enqueued) and a
// cleared control block.
struct ReplicaTables {
  unsigned long long t[48];
};
__global__ void k_replica_setup(Ctrl* ctl, unsigned long long* table, VolumeArgs* vol,
                                ReplicaTables t, VolumeArgs va) {
  if (blockIdx.x != 0) return;
  for (int i = threadIdx.x; i < 48; i += blockDim.x) table[i] = t.t[i];
  unsigned char* c = reinterpret_cast<unsigned char*>(ctl);
  for (int i = threadIdx.x; i < (int)sizeof(Ctrl); i += blockDim.x) c[i] = 0;
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&va);
  unsigned long long* dst = reinterpret_cast<unsigned long long*>(vol);
  for (int i = threadIdx.x; i < (int)(sizeof(VolumeArgs) / 8); i += blockDim.x) dst[i] = src[i];
}

__global__ void k_batch_reset(BatchWork* W, unsigned int* progress, int n_replicas) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_replicas; i += gridDim.x * blockDim.x)
    progress[i] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    W->next = 0;
    W->error = 0;
  }
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
template <int RNG_WORDS, bool CMP64, int TR, int TW>
__global__ void __launch_bounds__(kThreads, kBatchBlocksPerSM) k_batch_sweep(const ReplicaDesc* __restrict__ reps,
                                                             BatchWork* W,
                                                             const int32_t* __restrict__ order,
                                                             const long long* __restrict__ tile_prefix,
                                                             unsigned int* progress) {
  __shared__ TileSmem<TR, TW> S;
  __shared__ Tables2 Tb;
  __shared__ int s_rep, s_tile, s_valid, s_staged, s_abort, s_last;
  __shared__ long long s_rel;
  __shared__ int n_rep, n_tile, n_valid, n_ready;
  __shared__ long long n_rel;
  __shared__ uint32_t s_q;
  __shared__ uint32_t s_hist4[4];
  __shared__ RoundKeys s_keys;  // the current replica's round keys (broadcast reads)
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
      if ((int)(threadIdx.x >> 5) == kThreads / 32 - 1) {
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
    StepView<KeysRound> v;
    v.src = reinterpret_cast<const uint32_t*>(R.state + (size_t)(step & 1) * N);
    v.dst = reinterpret_cast<uint32_t*>(R.state + (size_t)((step + 1) & 1) * N);
    v.L = L;
    v.Lh = Lh;
    v.q = R.q;
    v.s_lo = (uint32_t)((unsigned long long)step & 0xFFFFFFFFu);
    v.s_hi = (uint32_t)((unsigned long long)step >> 32);
    v.keys.K = &s_keys;
    v.err = &W->error;
    const TileGeom gm = tile_geom<TR, TW>(L, Lh, (t / tiles_x) * TR, (t % tiles_x) * TW);
    if (staged)
      cp_async_wait_all();
    else
      stage_plain<TR, TW, kThreads, true>(v, gm, S);
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
    TileCounts cnt{0, 0, 0};
    const bool rec = step_recorded(vc->record_every, step);
    colour0<RNG_WORDS, CMP64, TR, TW, kThreads, kBatchShape>(v, gm, S, Tb, cnt, rec ? s_hist4 : nullptr);
    // S.in is free: take the next item and, when it can start, copy its tile.
    // The last warp takes it: it has the fewest rows (and no ring cells) in
    // the first colour, so the take overlaps the other warps' remaining work.
    if ((int)(threadIdx.x >> 5) == kThreads / 32 - 1) {
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
      stage_async16<TR, TW, kThreads>(vn, gn, S);
    }
    colour1<RNG_WORDS, CMP64, TR, TW, kThreads, kBatchShape>(v, gm, S, Tb, cnt, rec ? s_hist4 : nullptr);
    if (rec) {  // block-uniform: only on recorded steps
      __syncthreads();
      hist_flush(s_hist4, ctl->acc_hist);
    }
    uint32_t dhb = (uint32_t)cnt.dhb(), dc = (uint32_t)cnt.dc(), nacc = cnt.nacc;
    block_sum3<kThreads>(dhb, dc, nacc);  // two's complement sums
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

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

struct TileConfig {
  int rows, words;
};
constexpr TileConfig kTileConfigs[] = {{64, 64}, {32, 32}, {32, 16}, {16, 16}};
constexpr int kNumTileConfigs = 4;
constexpr long long kReplicaRingCap = 1024;
constexpr int kObsSlots = 4;  // observables tickets in flight per batch

struct Replica {
  bool live;
  cvf_params p;
  long long N;
  void* mem;  // one allocation: state pair, Ctrl, table, VolumeArgs, ring
  uint16_t* state;
  Ctrl* ctrl;
  unsigned long long* table;
  VolumeArgs* vol;
  cvf_obs* ring;
  long long ring_tail;
  long long sweep_host;
  bool cmp64;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct cvf_batch {
  cudaStream_t stream;
  cudaStream_t cap_stream;
  // replica memory and the descriptor array come from the batch's own
  // stream-ordered pool: a removed replica's memory is reused by a later
  // add on the same stream without a device-wide wait, and the pool keeps
  // what it has mapped until the batch is destroyed
  cudaMemPool_t pool;
  std::vector<Replica> reps;
  int rng_words;       // shared by all replicas (-1 while empty)
  int tile_cfg;        // -1: chosen per call
  int last_cfg;        // the shape the last call used
  ReplicaDesc* d_reps;
  int d_reps_cap;
  bool reps_dirty;
  void* d_work;
  size_t d_work_bytes;
  // pinned staging of the launch description and of the replica
  // descriptors, two slots each: a slot is rewritten only after the copy
  // that read it last has run (its event), so no call waits for a launch
  void* h_work[2];
  size_t h_work_bytes;
  cudaEvent_t ev_work[2];
  int work_slot;
  ReplicaDesc* h_descs[2];
  cudaEvent_t ev_descs[2];
  int descs_slot;
  // observables read-back: tickets rotate over kObsSlots slots, each with
  // device staging (records + histograms), a pinned copy of the records and
  // of the launch error word, and the event that marks the copy done
  struct ObsSlot {
    cvf_obs* d_obs;
    unsigned long long* d_hist;
    cvf_obs* h_obs;
    unsigned int* h_err;
    int cap;
    int n;
    long long ticket;
    cudaEvent_t ev;
  } obs[kObsSlots];
  long long next_ticket;
  void* h_pinned;     // 4096 bytes
  cudaGraphExec_t graph[kNumTileConfigs][2];  // [config][cmp64]
  int graph_n_reps[kNumTileConfigs][2];
  void* graph_work[kNumTileConfigs][2];
  int grid[kNumTileConfigs][2];
};

namespace {

using KernelFn = void (*)(const ReplicaDesc*, BatchWork*, const int32_t*, const long long*,
                          unsigned int*);

template <int RW, bool C64>
KernelFn pick_cfg(int cfg) {
  switch (cfg) {
    case 0: return k_batch_sweep<RW, C64, 64, 64>;
    case 1: return k_batch_sweep<RW, C64, 32, 32>;
    case 2: return k_batch_sweep<RW, C64, 32, 16>;
    default: return k_batch_sweep<RW, C64, 16, 16>;
  }
}

KernelFn pick_kernel(int rng_words, bool cmp64, int cfg) {
  if (rng_words == 1) return cmp64 ? pick_cfg<1, true>(cfg) : pick_cfg<1, false>(cfg);
  return cmp64 ? pick_cfg<2, true>(cfg) : pick_cfg<2, false>(cfg);
}

long long tiles_of(int L, int cfg) {
  const TileConfig& c = kTileConfigs[cfg];
  return (long long)((L / 2 + c.words - 1) / c.words) * ((L + c.rows - 1) / c.rows);
}

bool any_cmp64(const cvf_batch* b) {
  for (const Replica& r : b->reps)
    if (r.live && r.cmp64) return true;
  return false;
}

// Stream-ordered free: the memory returns to the pool once the work
// enqueued before it on the batch's stream is done (no device-wide wait).
void free_replica(Replica& r, cudaStream_t s) {
  if (r.mem) cudaFreeAsync(r.mem, s);
  r = Replica();
}

// Captured graphs hold device addresses; drop them when a buffer moves.
void drop_graphs(cvf_batch* b) {
  for (int c = 0; c < kNumTileConfigs; ++c)
    for (int k = 0; k < 2; ++k) {
      if (b->graph[c][k]) cudaGraphExecDestroy(b->graph[c][k]);
      b->graph[c][k] = nullptr;
    }
}

int upload_descs(cvf_batch* b) {
  if (!b->reps_dirty) return CVF_OK;
  const int n = (int)b->reps.size();
  if (n > b->d_reps_cap) {
    int cap = std::max(16, b->d_reps_cap * 2);
    while (cap < n) cap *= 2;
    ReplicaDesc* d = nullptr;
    CVF_CUDA_CHECK(cudaMallocFromPoolAsync(reinterpret_cast<void**>(&d), sizeof(ReplicaDesc) * cap,
                                           b->pool, b->stream));
    if (b->d_reps) CVF_CUDA_CHECK(cudaFreeAsync(b->d_reps, b->stream));
    // the staging slots grow with the descriptor array (after their copies)
    for (int k = 0; k < 2; ++k) {
      CVF_CUDA_CHECK(cudaEventSynchronize(b->ev_descs[k]));
      if (b->h_descs[k]) cudaFreeHost(b->h_descs[k]);
      b->h_descs[k] = nullptr;
      CVF_CUDA_CHECK(cudaMallocHost(reinterpret_cast<void**>(&b->h_descs[k]),
                                    sizeof(ReplicaDesc) * cap));
    }
    drop_graphs(b);
    b->d_reps = d;
    b->d_reps_cap = cap;
  }
  const int slot = b->descs_slot;
  b->descs_slot ^= 1;
  CVF_CUDA_CHECK(cudaEventSynchronize(b->ev_descs[slot]));  // the slot's last copy has run
  ReplicaDesc* h = b->h_descs[slot];
  for (int i = 0; i < n; ++i) {
    const Replica& r = b->reps[i];
    ReplicaDesc& d = h[i];
    std::memset(&d, 0, sizeof(d));
    if (!r.live) continue;
    d.state = r.state;
    d.ctrl = r.ctrl;
    d.table24 = r.table;
    d.vol = r.vol;
    d.ring = r.ring;
    d.ring_cap = kReplicaRingCap;
    d.keys = make_round_keys(r.p.seed);
    d.L = r.p.L;
    d.q = (uint32_t)r.p.q;
  }
  if (n > 0)
    CVF_CUDA_CHECK(cudaMemcpyAsync(b->d_reps, h, sizeof(ReplicaDesc) * n, cudaMemcpyHostToDevice,
                                   b->stream));
  CVF_CUDA_CHECK(cudaEventRecord(b->ev_descs[slot], b->stream));
  b->reps_dirty = false;
  return CVF_OK;
}

int ensure_work_buffer(cvf_batch* b, size_t bytes) {
  if (bytes <= b->d_work_bytes) return CVF_OK;
  size_t cap = std::max<size_t>(bytes, 2 * b->d_work_bytes);
  CVF_CUDA_CHECK(cudaStreamSynchronize(b->stream));  // growth only: rare
  if (b->d_work) cudaFree(b->d_work);
  for (int k = 0; k < 2; ++k) {
    if (b->h_work[k]) cudaFreeHost(b->h_work[k]);
    b->h_work[k] = nullptr;
  }
  b->d_work = nullptr;
  b->d_work_bytes = b->h_work_bytes = 0;
  drop_graphs(b);
  CVF_CUDA_CHECK(cudaMalloc(&b->d_work, cap));
  for (int k = 0; k < 2; ++k) CVF_CUDA_CHECK(cudaMallocHost(&b->h_work[k], cap));
  b->d_work_bytes = b->h_work_bytes = cap;
  return CVF_OK;
}

// Addresses of the arrays that follow the BatchWork header.
struct WorkLayout {
  size_t order_off, prefix_off, progress_off, total;
};
WorkLayout work_layout(int n_active, int n_reps) {
  WorkLayout w;
  w.order_off = align256(sizeof(BatchWork));
  w.prefix_off = align256(w.order_off + sizeof(int32_t) * std::max(n_active, 1));
  w.progress_off = align256(w.prefix_off + sizeof(long long) * (n_active + 1));
  w.total = align256(w.progress_off + sizeof(unsigned int) * std::max(n_reps, 1));
  return w;
}

// One launch over the work in b->d_work: reset + persistent kernel, captured
// as a graph the first time for a given configuration and replica count.
// Co-resident blocks of the kernel for a tile shape (the launch's grid).
int resident_grid(cvf_batch* b, int cfg, bool cmp64, int* grid) {
  const int c64 = cmp64 ? 1 : 0;
  if (b->grid[cfg][c64] == 0) {
    int per_sm = 0;
    KernelFn fn = pick_kernel(b->rng_words, cmp64, cfg);
    CVF_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn, kThreads, 0));
    if (per_sm < 1) return set_error(CVF_ECUDA, "batch kernel cannot be resident");
    b->grid[cfg][c64] = per_sm * sm_count();
  }
  *grid = b->grid[cfg][c64];
  return CVF_OK;
}

// The automatic tile shape of a call: the largest whose tiles over the
// advanced replicas give every co-resident block a tile per step.
int auto_tile_config(cvf_batch* b, const std::vector<int32_t>& act, bool cmp64, int* cfg) {
  for (int c = 0; c < kNumTileConfigs; ++c) {
    int grid = 0;
    const int rc = resident_grid(b, c, cmp64, &grid);
    if (rc) return rc;
    long long tiles = 0;
    for (int i : act) tiles += tiles_of(b->reps[i].p.L, c);
    if (tiles >= grid) {
      *cfg = c;
      return CVF_OK;
    }
  }
  *cfg = kNumTileConfigs - 1;
  return CVF_OK;
}

int launch(cvf_batch* b, int cfg, bool cmp64, int n_reps, int n_active) {
  const int c64 = cmp64 ? 1 : 0;
  KernelFn fn = pick_kernel(b->rng_words, cmp64, cfg);
  int grid_unused = 0;
  int grc = resident_grid(b, cfg, cmp64, &grid_unused);
  if (grc) return grc;
  (void)n_active;
  const WorkLayout wl = work_layout(n_reps, n_reps);
  char* base = reinterpret_cast<char*>(b->d_work);
  BatchWork* W = reinterpret_cast<BatchWork*>(base);
  const int32_t* order = reinterpret_cast<const int32_t*>(base + wl.order_off);
  const long long* prefix = reinterpret_cast<const long long*>(base + wl.prefix_off);
  unsigned int* progress = reinterpret_cast<unsigned int*>(base + wl.progress_off);
  auto enqueue = [&](cudaStream_t s) -> cudaError_t {
    k_batch_reset<<<std::max(1, (n_reps + 255) / 256), 256, 0, s>>>(W, progress, n_reps);
    cudaLaunchConfig_t lc;
    std::memset(&lc, 0, sizeof(lc));
    lc.gridDim = dim3(b->grid[cfg][c64]);
    lc.blockDim = dim3(kThreads);
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, fn, (const ReplicaDesc*)b->d_reps, W, order, prefix, progress);
  };
  // the graph bakes in the array offsets, which depend on the counts
  const bool reuse = b->graph[cfg][c64] && b->graph_n_reps[cfg][c64] == n_reps &&
                     b->graph_work[cfg][c64] == b->d_work;
  if (!reuse) {
    if (b->graph[cfg][c64]) {
      cudaGraphExecDestroy(b->graph[cfg][c64]);
      b->graph[cfg][c64] = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = enqueue(b->cap_stream);
      e = cudaStreamEndCapture(b->cap_stream, &g);
      if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) {
      e = cudaGraphInstantiate(&b->graph[cfg][c64], g, 0);
      cudaGraphDestroy(g);
    }
    if (e != cudaSuccess) {
      b->graph[cfg][c64] = nullptr;
      cudaGetLastError();
      // capture unsupported here: launch directly (still one persistent launch)
      CVF_CUDA_CHECK(enqueue(b->stream));
      return CVF_OK;
    }
    b->graph_n_reps[cfg][c64] = n_reps;
    b->graph_work[cfg][c64] = b->d_work;
  }
  CVF_CUDA_CHECK(cudaGraphLaunch(b->graph[cfg][c64], b->stream));
  return CVF_OK;
}

int check_replica(cvf_batch* b, int32_t id) {
  if (!b) return set_error(CVF_EINVAL, "batch is NULL");
  if (id < 0 || id >= (int)b->reps.size() || !b->reps[id].live)
    return set_error(CVF_EINVAL, "replica %d does not exist", id);
  return CVF_OK;
}

int launch_error(unsigned int err) {
  if (err >= 0x100u)
    return set_error(CVF_EBOUNDS, "a device index check of the batched sweep failed (site %u)",
                     err - 0x100u);
  if (err) return set_error(CVF_ETIMEOUT, "a replica wait in the batched sweep gave up");
  return CVF_OK;
}

// (Re)allocates a ticket slot's staging for cap records; the slot's last
// copy must be done.
cudaError_t grow_obs_slot(cvf_batch::ObsSlot& o, int cap) {
  if (o.d_obs) cudaFree(o.d_obs);
  if (o.d_hist) cudaFree(o.d_hist);
  if (o.h_obs) cudaFreeHost(o.h_obs);
  o.d_obs = nullptr;
  o.d_hist = nullptr;
  o.h_obs = nullptr;
  o.cap = 0;
  cudaError_t e = cudaMalloc(&o.d_obs, sizeof(cvf_obs) * cap);
  if (e == cudaSuccess) e = cudaMalloc(&o.d_hist, sizeof(unsigned long long) * 9 * cap);
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&o.h_obs), sizeof(cvf_obs) * cap);
  if (e == cudaSuccess) o.cap = cap;
  return e;
}

// Reads the error word of the last launch (synchronises the stream).
int batch_status(cvf_batch* b) {
  CVF_CUDA_CHECK(cudaStreamSynchronize(b->stream));
  if (!b->d_work) return CVF_OK;
  CVF_CUDA_CHECK(cudaMemcpyAsync(b->h_pinned,
                                 reinterpret_cast<char*>(b->d_work) + offsetof(BatchWork, error),
                                 sizeof(unsigned int), cudaMemcpyDeviceToHost, b->stream));
  CVF_CUDA_CHECK(cudaStreamSynchronize(b->stream));
  unsigned int err = 0;
  std::memcpy(&err, b->h_pinned, sizeof(err));
  return launch_error(err);
}

}  // namespace

extern "C" {

int cvf_batch_create(const cvf_params* params, int32_t n, void* stream, cvf_batch** out) {
  NvtxRange nvtx_range("cvf_batch_create");
  if (!out) return set_error(CVF_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 0 || (n > 0 && !params)) return set_error(CVF_EINVAL, "bad replica list");
  cvf_batch* b = new (std::nothrow) cvf_batch();
  if (!b) return set_error(CVF_ENOMEM, "host allocation failed");
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  b->rng_words = -1;
  b->tile_cfg = -1;
  b->last_cfg = -1;
  cudaError_t e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    int dev = 0;
    e = cudaGetDevice(&dev);
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (e == cudaSuccess) e = cudaMemPoolCreate(&b->pool, &props);
    uint64_t keep = ~0ull;
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(b->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_pinned, 4096);
  for (int k = 0; k < kObsSlots && e == cudaSuccess; ++k) {
    b->obs[k].ticket = -1;
    e = cudaEventCreateWithFlags(&b->obs[k].ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&b->obs[k].h_err), 64);
    if (e == cudaSuccess) e = grow_obs_slot(b->obs[k], 16);
  }
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&b->ev_work[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_descs[k], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    cvf_batch_destroy(b);
    return set_error(CVF_ECUDA, "batch setup: %s", cudaGetErrorString(e));
  }
  for (int i = 0; i < n; ++i) {
    int32_t id;
    const int rc = cvf_batch_add(b, &params[i], &id);
    if (rc) {
      cvf_batch_destroy(b);
      return rc;
    }
  }
  *out = b;
  return CVF_OK;
}

int cvf_batch_add(cvf_batch* b, const cvf_params* p, int32_t* replica) {
  NvtxRange nvtx_range("cvf_batch_add");
  if (!b || !replica) return set_error(CVF_EINVAL, "NULL argument");
  int rc = check_params(p);
  if (rc) return rc;
  if (p->schedule != CVF_SCHED_CHECKERBOARD)
    return set_error(CVF_EINVAL, "batched replicas use the checkerboard schedule");
  if (b->rng_words >= 0 && p->rng_words != b->rng_words)
    return set_error(CVF_EINVAL, "all replicas of a batch share rng_words (%d)", b->rng_words);
  std::vector<int64_t> d2, mult;
  lattice_shells(p->cutoff, &d2, &mult);
  if ((int)d2.size() > kMaxShells) return set_error(CVF_EINVAL, "cutoff too large");
  Replica r = Replica();
  r.p = *p;
  r.N = (long long)p->L * p->L;
  const size_t o_state = 0;
  const size_t o_ctrl = align256(o_state + sizeof(uint16_t) * 2 * (size_t)r.N);
  const size_t o_table = align256(o_ctrl + sizeof(Ctrl));
  const size_t o_vol = align256(o_table + sizeof(unsigned long long) * 48);
  const size_t o_ring = align256(o_vol + sizeof(VolumeArgs));
  const size_t total = align256(o_ring + sizeof(cvf_obs) * kReplicaRingCap);
  cudaError_t e = cudaMallocFromPoolAsync(&r.mem, total, b->pool, b->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(e == cudaErrorMemoryAllocation ? CVF_ENOMEM : CVF_ECUDA,
                     "replica allocation (%zu bytes): %s", total, cudaGetErrorString(e));
  }
  char* m = reinterpret_cast<char*>(r.mem);
  r.state = reinterpret_cast<uint16_t*>(m + o_state);
  r.ctrl = reinterpret_cast<Ctrl*>(m + o_ctrl);
  r.table = reinterpret_cast<unsigned long long*>(m + o_table);
  r.vol = reinterpret_cast<VolumeArgs*>(m + o_vol);
  r.ring = reinterpret_cast<cvf_obs*>(m + o_ring);
  ReplicaTables t24;
  r.cmp64 = fill_table24(p, t24.t);
  VolumeArgs va;
  fill_volume_args(p, r.N, d2, mult, &va);
  const RoundKeys K = make_round_keys(p->seed);
  cudaStream_t s = b->stream;
#define ADD_CHECK(expr)                                                             \
  do {                                                                              \
    cudaError_t e_ = (expr);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      free_replica(r, s);                                                           \
      return set_error(CVF_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_)); \
    }                                                                               \
  } while (0)
  // everything is enqueued on the batch's stream (after any launch in
  // flight) and the host data travel as kernel parameters: no wait here
  k_replica_setup<<<1, 256, 0, s>>>(r.ctrl, r.table, r.vol, t24, va);
  const int grid = (int)std::max<long long>(1, std::min<long long>((r.N + 255) / 256, 4096));
  k_init<<<grid, 256, 0, s>>>(r.state, p->L, (uint32_t)p->q, p->init == CVF_INIT_RANDOM ? 1 : 0, K);
  k_set_ctrl<<<1, 32, 0, s>>>(r.vol, r.ctrl, (double)r.N * p->v_iso_init, 0, r.N);
  k_recount<<<grid, kThreads, 0, s>>>(r.state, p->L, nullptr, &r.ctrl->acc_hb);
  k_commit_counts<<<1, 32, 0, s>>>(r.ctrl);
  k_volume_prologue<<<1, 32, 0, s>>>(r.vol, r.ctrl, K);
  ADD_CHECK(cudaGetLastError());
#undef ADD_CHECK
  r.live = true;
  r.sweep_host = 0;
  r.ring_tail = 0;
  int id = -1;
  for (int i = 0; i < (int)b->reps.size(); ++i)
    if (!b->reps[i].live) {
      id = i;
      break;
    }
  if (id < 0) {
    id = (int)b->reps.size();
    b->reps.push_back(r);
  } else {
    b->reps[id] = r;
  }
  if (b->rng_words < 0) b->rng_words = p->rng_words;
  b->reps_dirty = true;
  *replica = id;
  return CVF_OK;
}

int cvf_batch_remove(cvf_batch* b, int32_t replica) {
  int rc = check_replica(b, replica);
  if (rc) return rc;
  // stream-ordered: the memory is released after the launches already
  // enqueued (which may still be reading it) have run
  free_replica(b->reps[replica], b->stream);
  CVF_CUDA_CHECK(cudaGetLastError());
  b->reps_dirty = true;
  bool any = false;
  for (const Replica& r : b->reps) any = any || r.live;
  if (!any) b->rng_words = -1;
  return CVF_OK;
}

int cvf_batch_size(cvf_batch* b, int32_t* n_slots, int32_t* n_live) {
  if (!b || !n_slots || !n_live) return set_error(CVF_EINVAL, "NULL argument");
  *n_slots = (int32_t)b->reps.size();
  int live = 0;
  for (const Replica& r : b->reps) live += r.live ? 1 : 0;
  *n_live = live;
  return CVF_OK;
}

int cvf_batch_set_tiles(cvf_batch* b, int32_t config) {
  if (!b) return set_error(CVF_EINVAL, "batch is NULL");
  if (config < -1 || config >= kNumTileConfigs)
    return set_error(CVF_EINVAL, "tile config %d (-1 automatic, 0..%d)", config,
                     kNumTileConfigs - 1);
  b->tile_cfg = config;
  return CVF_OK;
}

int cvf_batch_get_tiles(cvf_batch* b, int32_t* config, int32_t* last_used) {
  if (!b || !config || !last_used) return set_error(CVF_EINVAL, "NULL argument");
  *config = b->tile_cfg;
  *last_used = b->last_cfg;
  return CVF_OK;
}

int cvf_batch_tile_config(int32_t config, int32_t* rows, int32_t* words) {
  if (config < 0 || config >= kNumTileConfigs || !rows || !words)
    return set_error(CVF_EINVAL, "tile config %d (0..%d)", config, kNumTileConfigs - 1);
  *rows = kTileConfigs[config].rows;
  *words = kTileConfigs[config].words;
  return CVF_OK;
}

int cvf_batch_sweep(cvf_batch* b, const int64_t* sweeps, int32_t n) {
  NvtxRange nvtx_range("cvf_batch_sweep");
  if (!b) return set_error(CVF_EINVAL, "batch is NULL");
  if (n != (int)b->reps.size() || (n > 0 && !sweeps))
    return set_error(CVF_EINVAL, "need one step count per replica slot (%zu)", b->reps.size());
  std::vector<int32_t> act;
  for (int i = 0; i < n; ++i) {
    if (sweeps[i] < 0) return set_error(CVF_EINVAL, "negative step count for replica %d", i);
    if (sweeps[i] > 0 && !b->reps[i].live)
      return set_error(CVF_EINVAL, "steps requested for removed replica %d", i);
    if (sweeps[i] > 0) act.push_back(i);
  }
  if (act.empty()) return CVF_OK;
  for (int i : act)
    if (sweeps[i] > 0x7FFFFFFF) return set_error(CVF_EINVAL, "at most 2^31-1 steps per call");
  int rc = upload_descs(b);
  if (rc) return rc;
  std::stable_sort(act.begin(), act.end(), [&](int a, int c) { return sweeps[a] > sweeps[c]; });
  int cfg = b->tile_cfg;
  if (cfg < 0) {
    rc = auto_tile_config(b, act, any_cmp64(b), &cfg);
    if (rc) return rc;
  }
  b->last_cfg = cfg;
  const int na = (int)act.size();
  // array capacities follow the slot count, so a captured graph stays valid
  // whatever subset of replicas a call advances
  const WorkLayout wl = work_layout(n, n);
  rc = ensure_work_buffer(b, wl.total);
  if (rc) return rc;
  // segments of constant active prefix, in increasing relative step
  std::vector<long long> prefix(na + 1, 0);
  // a replica-step's items: its tiles and one volume item (the next step's move)
  for (int k = 0; k < na; ++k)
    prefix[k + 1] = prefix[k] + tiles_of(b->reps[act[k]].p.L, cfg) + 1;
  std::vector<long long> bounds;  // distinct step counts, ascending
  for (int k = na - 1; k >= 0; --k)
    if (bounds.empty() || bounds.back() != sweeps[act[k]]) bounds.push_back(sweeps[act[k]]);
  if ((int)bounds.size() > kBatchMaxSegments)
    return set_error(CVF_EINVAL, "at most %d distinct step counts per call", kBatchMaxSegments);
  // the description goes through one of two pinned slots; a slot is
  // rewritten once the copy that read it two calls ago has run
  const int slot = b->work_slot;
  b->work_slot ^= 1;
  CVF_CUDA_CHECK(cudaEventSynchronize(b->ev_work[slot]));
  char* h = reinterpret_cast<char*>(b->h_work[slot]);
  std::memset(h, 0, sizeof(BatchWork));
  BatchWork* W = reinterpret_cast<BatchWork*>(h);
  W->n_active = na;
  W->tile_rows = kTileConfigs[cfg].rows;
  W->tile_words = kTileConfigs[cfg].words;
  long long s0 = 0, base = 0;
  int nseg = 0;
  for (long long ub : bounds) {
    int active = 0;
    while (active < na && sweeps[act[active]] > s0) ++active;
    W->seg_s0[nseg] = s0;
    W->seg_base[nseg] = base;
    W->seg_active[nseg] = active;
    base += (ub - s0) * prefix[active];
    s0 = ub;
    ++nseg;
  }
  W->seg_s0[nseg] = s0;
  W->seg_base[nseg] = base;
  W->nseg = nseg;
  W->total_items = base;
  std::memcpy(h + wl.order_off, act.data(), sizeof(int32_t) * na);
  std::memcpy(h + wl.prefix_off, prefix.data(), sizeof(long long) * (na + 1));
  CVF_CUDA_CHECK(cudaMemcpyAsync(b->d_work, h, wl.progress_off, cudaMemcpyHostToDevice, b->stream));
  CVF_CUDA_CHECK(cudaEventRecord(b->ev_work[slot], b->stream));
  rc = launch(b, cfg, any_cmp64(b), n, na);
  if (rc) return rc;
  for (int i : act) b->reps[i].sweep_host += sweeps[i];
  return CVF_OK;
}

int cvf_batch_sync(cvf_batch* b) {
  NvtxRange nvtx_range("cvf_batch_sync");
  if (!b) return set_error(CVF_EINVAL, "batch is NULL");
  return batch_status(b);
}

int cvf_batch_observables_enqueue(cvf_batch* b, const int32_t* replicas, int32_t n,
                                  int64_t* ticket) {
  NvtxRange nvtx_range("cvf_batch_observables_enqueue");
  if (!b || !ticket || n < 0 || (n > 0 && !replicas)) return set_error(CVF_EINVAL, "bad argument");
  for (int i = 0; i < n; ++i) {
    const int rc = check_replica(b, replicas[i]);
    if (rc) return rc;
  }
  const long long t = b->next_ticket;
  cvf_batch::ObsSlot& o = b->obs[t % kObsSlots];
  // the slot's previous ticket (kObsSlots enqueues ago) has been copied out
  // by now or is given up
  CVF_CUDA_CHECK(cudaEventSynchronize(o.ev));
  if (n > o.cap) {
    int cap = o.cap;
    while (cap < n) cap *= 2;
    CVF_CUDA_CHECK(grow_obs_slot(o, cap));
  }
  if (n > 0) {
    CVF_CUDA_CHECK(cudaMemsetAsync(o.d_hist, 0, sizeof(unsigned long long) * 9 * n, b->stream));
    for (int i = 0; i < n; ++i) {
      const Replica& r = b->reps[replicas[i]];
      const int grid = (int)std::max<long long>(1, std::min<long long>((r.N + kThreads - 1) / kThreads, 2048));
      k_histogram<<<grid, kThreads, 0, b->stream>>>(r.state + (size_t)(r.sweep_host & 1) * r.N, r.N,
                                                    o.d_hist + 9 * i);
      k_observables<<<1, 32, 0, b->stream>>>(r.vol, r.ctrl, o.d_hist + 9 * i, o.d_obs + i);
    }
    CVF_CUDA_CHECK(cudaGetLastError());
    CVF_CUDA_CHECK(cudaMemcpyAsync(o.h_obs, o.d_obs, sizeof(cvf_obs) * n, cudaMemcpyDeviceToHost,
                                   b->stream));
  }
  o.h_err[0] = 0;
  if (b->d_work)
    CVF_CUDA_CHECK(cudaMemcpyAsync(o.h_err, reinterpret_cast<char*>(b->d_work) + offsetof(BatchWork, error),
                                   sizeof(unsigned int), cudaMemcpyDeviceToHost, b->stream));
  CVF_CUDA_CHECK(cudaEventRecord(o.ev, b->stream));
  o.n = n;
  o.ticket = t;
  b->next_ticket = t + 1;
  *ticket = t;
  return CVF_OK;
}

int cvf_batch_observables_collect(cvf_batch* b, int64_t ticket, cvf_obs* out, int32_t n) {
  NvtxRange nvtx_range("cvf_batch_observables_collect");
  if (!b || n < 0 || (n > 0 && !out) || ticket < 0) return set_error(CVF_EINVAL, "bad argument");
  cvf_batch::ObsSlot& o = b->obs[ticket % kObsSlots];
  if (o.ticket != ticket)
    return set_error(CVF_EINVAL, "ticket %lld was overwritten (at most %d in flight)",
                     (long long)ticket, kObsSlots);
  if (n != o.n) return set_error(CVF_EINVAL, "ticket %lld holds %d records, not %d",
                                 (long long)ticket, o.n, n);
  CVF_CUDA_CHECK(cudaEventSynchronize(o.ev));  // waits up to this point of the stream only
  const int rc = launch_error(o.h_err[0]);
  if (rc) return rc;
  if (n > 0) std::memcpy(out, o.h_obs, sizeof(cvf_obs) * n);
  return CVF_OK;
}

int cvf_batch_observables_many(cvf_batch* b, const int32_t* replicas, int32_t n, cvf_obs* out) {
  NvtxRange nvtx_range("cvf_batch_observables_many");
  int64_t t = -1;
  int rc = cvf_batch_observables_enqueue(b, replicas, n, &t);
  if (rc) return rc;
  return cvf_batch_observables_collect(b, t, out, n);
}

int cvf_batch_observables(cvf_batch* b, int32_t replica, cvf_obs* out) {
  NvtxRange nvtx_range("cvf_batch_observables");
  if (!out) return set_error(CVF_EINVAL, "out is NULL");
  return cvf_batch_observables_many(b, &replica, 1, out);
}

int cvf_batch_get_state(cvf_batch* b, int32_t replica, uint16_t* host, size_t n) {
  NvtxRange nvtx_range("cvf_batch_get_state");
  int rc = check_replica(b, replica);
  if (rc) return rc;
  const Replica& r = b->reps[replica];
  if (!host || (long long)n != r.N)
    return set_error(CVF_EINVAL, "n=%zu, replica %d has %lld cells", n, replica, r.N);
  rc = batch_status(b);
  if (rc) return rc;
  CVF_CUDA_CHECK(cudaMemcpyAsync(host, r.state + (size_t)(r.sweep_host & 1) * r.N,
                                 sizeof(uint16_t) * n, cudaMemcpyDeviceToHost, b->stream));
  CVF_CUDA_CHECK(cudaStreamSynchronize(b->stream));
  return CVF_OK;
}

int cvf_batch_memory(cvf_batch* b, uint64_t* reserved, uint64_t* used) {
  if (!b || !reserved || !used) return set_error(CVF_EINVAL, "NULL argument");
  unsigned long long r = 0, u = 0;  // 64-bit values, as the attributes are
  CVF_CUDA_CHECK(cudaMemPoolGetAttribute(b->pool, cudaMemPoolAttrReservedMemCurrent, &r));
  CVF_CUDA_CHECK(cudaMemPoolGetAttribute(b->pool, cudaMemPoolAttrUsedMemCurrent, &u));
  *reserved = (uint64_t)r;
  *used = (uint64_t)u;
  return CVF_OK;
}

int cvf_batch_destroy(cvf_batch* b) {
  if (!b) return CVF_OK;
  for (Replica& r : b->reps) free_replica(r, b->stream);
  if (b->d_reps) cudaFreeAsync(b->d_reps, b->stream);
  b->d_reps = nullptr;
  cudaStreamSynchronize(b->stream);
  for (int c = 0; c < kNumTileConfigs; ++c)
    for (int k = 0; k < 2; ++k)
      if (b->graph[c][k]) cudaGraphExecDestroy(b->graph[c][k]);
  if (b->d_work) cudaFree(b->d_work);
  for (int k = 0; k < 2; ++k) {
    if (b->h_work[k]) cudaFreeHost(b->h_work[k]);
    if (b->h_descs[k]) cudaFreeHost(b->h_descs[k]);
    if (b->ev_work[k]) cudaEventDestroy(b->ev_work[k]);
    if (b->ev_descs[k]) cudaEventDestroy(b->ev_descs[k]);
  }
  for (int k = 0; k < kObsSlots; ++k) {
    cvf_batch::ObsSlot& o = b->obs[k];
    if (o.d_obs) cudaFree(o.d_obs);
    if (o.d_hist) cudaFree(o.d_hist);
    if (o.h_obs) cudaFreeHost(o.h_obs);
    if (o.h_err) cudaFreeHost(o.h_err);
    if (o.ev) cudaEventDestroy(o.ev);
  }
  if (b->h_pinned) cudaFreeHost(b->h_pinned);
  if (b->pool) cudaMemPoolDestroy(b->pool);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  delete b;
  return CVF_OK;
}

}  // extern "C"
