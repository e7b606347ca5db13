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
      w = __umulhi(r.x, q) | (__umulhi(r.y, q) << 3) | (__umulhi(r.z, q) << 6) |
          (__umulhi(r.w, q) << 9);
    }
    state[c] = (uint16_t)w;
  }
}

// Full recount of N_HB_raw (the +x and +y bond of every cell) and N_sigma
// (equal pairs inside every cell); adds the totals to out[0], out[1].
__global__ void __launch_bounds__(kThreads) k_recount(const uint16_t* __restrict__ state,
                                                      int32_t L,
                                                      unsigned long long* out) {
  const long long N = (long long)L * L;
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

__global__ void k_set_ctrl(Ctrl* ctl, double V_iso, long long sweep, long long N) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl->sweep = sweep;
    ctl->V_iso = V_iso;
    ctl->g = (V_iso / (double)N < 2.0) ? 1 : 0;
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

// One volume move (single thread).
__global__ void k_volume_move(const VolumeArgs* __restrict__ V, Ctrl* ctl, RoundKeys K) {
  if (threadIdx.x == 0 && blockIdx.x == 0) volume_move(*V, ctl, K);
}

__global__ void k_observables(const VolumeArgs* __restrict__ V, const Ctrl* ctl,
                              cvf_obs* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = make_obs(*V, ctl);
}

// End of a step, run by one thread once every block's counts are in:
// commit the counts, advance the step counter, append the observables to the
// ring when the step count is a multiple of record_every.
__device__ __forceinline__ void finalize_step(const VolumeArgs& V, Ctrl* ctl, cvf_obs* ring,
                                              long long ring_cap) {
  volatile Ctrl* vc = ctl;
  const unsigned long long hb = vc->acc_hb, pairs = vc->acc_pairs, moves = vc->acc_moves;
  ctl->n_hb_raw = (long long)hb;
  ctl->n_coop = (long long)pairs;
  ctl->acc_sigma += (long long)moves;
  ctl->acc_hb = 0;
  ctl->acc_pairs = 0;
  ctl->acc_moves = 0;
  ctl->done = 0;
  ctl->sweep += 1;
  const int every = ctl->record_every;
  if (every > 0 && ctl->sweep % every == 0) {
    ring[ctl->ring_head % ring_cap] = make_obs(V, ctl);
    ctl->ring_head += 1;
  }
}

// True in every thread of the block that arrives last (after all blocks
// have published their atomics).
__device__ __forceinline__ bool last_block(unsigned int* done) {
  __shared__ int is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int prev = atomicAdd(done, 1u);
    is_last = (prev == gridDim.x - 1) ? 1 : 0;
    if (is_last) __threadfence();
  }
  __syncthreads();
  return is_last != 0;
}

// Checkerboard half-sweep (colour k): every cell with (x + y) & 1 == k updates
// its four arms.  Cells of one colour interact only through cells of the
// other colour, which stay fixed during the half-sweep, so the update is in
// place.  One thread handles one 32-bit word = a pair of horizontally
// adjacent cells, exactly one of which has colour k.  Colour 0 adds the
// in-cell pair counts of its cells; colour 1 adds those of its cells and the
// bonds of its cells (every bond has exactly one colour-1 end) and, in the
// last block, closes the step.
template <int RNG_WORDS>
__global__ void __launch_bounds__(kThreads) k_half_sweep(LatticeArgs A, int colour) {
  __shared__ unsigned long long sT[21];
  Ctrl* ctl = A.ctrl;
  const int g = ctl->g;
  const long long step = ctl->sweep;
  if (threadIdx.x < 21) sT[threadIdx.x] = A.table[g * 21 + threadIdx.x];
  __syncthreads();
  const uint32_t s_lo = (uint32_t)((unsigned long long)step & 0xFFFFFFFFu);
  const uint32_t s_hi = (uint32_t)((unsigned long long)step >> 32);
  const int L = A.L;
  const int Lh = L >> 1;
  const long long npairs = (long long)L * Lh;
  const uint32_t* __restrict__ st32 = reinterpret_cast<const uint32_t*>(A.state);
  uint32_t pairs = 0, bonds = 0, nacc = 0;
  for (long long pi = blockIdx.x * (long long)blockDim.x + threadIdx.x; pi < npairs;
       pi += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(pi / Lh);
    const int p = (int)(pi - (long long)y * Lh);
    const int hi = (y + colour) & 1;  // own cell in the high half of the word
    const int x = 2 * p + hi;
    const uint32_t own = st32[pi];
    const uint32_t wyp = st32[(long long)(y + 1 == L ? 0 : y + 1) * Lh + p];
    const uint32_t wym = st32[(long long)(y == 0 ? L - 1 : y - 1) * Lh + p];
    uint32_t w, nxp, nxm;
    if (hi) {
      w = own >> 16;
      nxm = own & 0xFFFFu;
      nxp = st32[(long long)y * Lh + (p + 1 == Lh ? 0 : p + 1)] & 0xFFFFu;
    } else {
      w = own & 0xFFFFu;
      nxp = own >> 16;
      nxm = st32[(long long)y * Lh + (p == 0 ? Lh - 1 : p - 1)] >> 16;
    }
    const uint32_t nyp = hi ? (wyp >> 16) : (wyp & 0xFFFFu);
    const uint32_t nym = hi ? (wym >> 16) : (wym & 0xFFFFu);
    // partner arms: arm 0 (+x) <-> arm 1 of the +x cell, arm 1 (-x) <-> arm 0
    // of the -x cell, arm 2 (+y) <-> arm 3 of the +y cell, arm 3 <-> arm 2
    const uint32_t part[4] = {arm_of(nxp, 1), arm_of(nxm, 0), arm_of(nyp, 3), arm_of(nym, 2)};
    uint32_t acc[4], kk[4];
    cell_draws<RNG_WORDS>((uint32_t)((long long)y * L + x), s_lo, s_hi, A.keys, A.q, acc, kk);
    w = update_cell(w, part, acc, kk, A.q, sT, nacc);
    A.state[(long long)y * L + x] = (uint16_t)w;
    pairs += cell_pairs(w);
    if (colour) bonds += cell_bonds(w, part);
  }
  block_sum3<kThreads>(pairs, bonds, nacc);
  if (threadIdx.x == 0) {
    atomicAdd(&ctl->acc_pairs, (unsigned long long)pairs);
    if (colour) atomicAdd(&ctl->acc_hb, (unsigned long long)bonds);
    atomicAdd(&ctl->acc_moves, (unsigned long long)nacc);
  }
  if (colour == 1 && last_block(&ctl->done) && threadIdx.x == 0)
    finalize_step(*A.vol, ctl, A.ring, A.ring_cap);
}

// Layered schedule: pass `pass` updates arm order[pass] of every cell, where
// the order is a Fisher-Yates permutation drawn from Philox((2^32-2, step,
// tag 4)).  The same arm of all cells forms one domain (its members interact
// only with other domains), so the pass is in place.
template <int RNG_WORDS>
__global__ void __launch_bounds__(kThreads) k_layer_pass(LatticeArgs A, int pass) {
  __shared__ unsigned long long sT[21];
  __shared__ int s_arm;
  Ctrl* ctl = A.ctrl;
  const int g = ctl->g;
  const long long step = ctl->sweep;
  const uint32_t s_lo = (uint32_t)((unsigned long long)step & 0xFFFFFFFFu);
  const uint32_t s_hi = (uint32_t)((unsigned long long)step >> 32);
  if (threadIdx.x < 21) sT[threadIdx.x] = A.table[g * 21 + threadIdx.x];
  if (threadIdx.x == 0) {
    const Words4 r = philox(kCellLayers, s_lo, s_hi, kTagLayers, A.keys);
    const uint32_t rw[4] = {r.x, r.y, r.z, r.w};
    int order[4] = {0, 1, 2, 3};
    for (int i = 3; i >= 1; --i) {
      const int j = (int)__umulhi(rw[3 - i], (uint32_t)(i + 1));
      const int t = order[i];
      order[i] = order[j];
      order[j] = t;
    }
    s_arm = order[pass];
  }
  __syncthreads();
  const int a = s_arm;
  const int L = A.L;
  const long long N = (long long)L * L;
  uint32_t nacc = 0, unused0 = 0, unused1 = 0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(c / L), x = (int)(c - (long long)y * L);
    int xn = x, yn = y;
    if (a == 0) xn = (x + 1 == L) ? 0 : x + 1;
    else if (a == 1) xn = (x == 0) ? L - 1 : x - 1;
    else if (a == 2) yn = (y + 1 == L) ? 0 : y + 1;
    else yn = (y == 0) ? L - 1 : y - 1;
    const uint32_t w = A.state[c];
    const uint32_t n = arm_of(A.state[(long long)yn * L + xn], a ^ 1);
    uint32_t acc[4], kk[4];
    cell_draws<RNG_WORDS>((uint32_t)c, s_lo, s_hi, A.keys, A.q, acc, kk);
    const uint32_t s = arm_of(w, a);
    uint32_t sp = s + 1u + kk[a];
    sp = (sp >= A.q) ? sp - A.q : sp;
    const int dhb = (int)(sp == n) - (int)(s == n);
    int dc = 0;
    for (int b = 0; b < 4; ++b) {
      if (b == a) continue;
      const uint32_t sb = arm_of(w, b);
      dc += (int)(sp == sb) - (int)(s == sb);
    }
    if ((unsigned long long)acc[a] < sT[(dhb + 1) * 7 + (dc + 3)]) {
      A.state[c] = (uint16_t)((w & ~(7u << (3 * a))) | (sp << (3 * a)));
      ++nacc;
    }
  }
  block_sum3<kThreads>(nacc, unused0, unused1);
  if (threadIdx.x == 0) atomicAdd(&ctl->acc_moves, (unsigned long long)nacc);
}

// Close a layered step after the recount of its final configuration.
__global__ void k_finalize(LatticeArgs A) {
  if (threadIdx.x == 0 && blockIdx.x == 0) finalize_step(*A.vol, A.ctrl, A.ring, A.ring_cap);
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
  unsigned long long* table_dev;
  VolumeArgs* vol_dev;
  unsigned long long* rc_dev;
  void* host_pinned;
  LatticeArgs args;
  int grid_pairs, grid_cells;
  cudaGraphExec_t graph;
  int graph_steps;
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

// Enqueue one MC step on stream s.
void enqueue_step(cvf_handle* h, cudaStream_t s) {
  if (h->p.volume_moves) k_volume_move<<<1, 32, 0, s>>>(h->vol_dev, h->ctrl, h->args.keys);
  const bool one = h->p.rng_words == 1;
  if (h->p.schedule == CVF_SCHED_CHECKERBOARD) {
    for (int colour = 0; colour < 2; ++colour) {
      if (one)
        k_half_sweep<1><<<h->grid_pairs, kThreads, 0, s>>>(h->args, colour);
      else
        k_half_sweep<2><<<h->grid_pairs, kThreads, 0, s>>>(h->args, colour);
    }
  } else {
    for (int pass = 0; pass < 4; ++pass) {
      if (one)
        k_layer_pass<1><<<h->grid_cells, kThreads, 0, s>>>(h->args, pass);
      else
        k_layer_pass<2><<<h->grid_cells, kThreads, 0, s>>>(h->args, pass);
    }
    k_recount<<<h->grid_cells, kThreads, 0, s>>>(h->state, h->p.L, &h->ctrl->acc_hb);
    k_finalize<<<1, 32, 0, s>>>(h->args);
  }
}

int recount_into_ctrl(cvf_handle* h) {
  // acc_hb and acc_pairs are adjacent: the recount adds into both
  static_assert(offsetof(Ctrl, acc_pairs) == offsetof(Ctrl, acc_hb) + 8, "layout");
  k_recount<<<h->grid_cells, kThreads, 0, h->stream>>>(h->state, h->p.L, &h->ctrl->acc_hb);
  k_commit_counts<<<1, 32, 0, h->stream>>>(h->ctrl);
  CVF_CUDA_CHECK(cudaGetLastError());
  return CVF_OK;
}

int build_graph(cvf_handle* h) {
  if (h->graph) return CVF_OK;
  cudaGraph_t g = nullptr;
  CVF_CUDA_CHECK(cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
  for (int i = 0; i < kGraphSteps; ++i) enqueue_step(h, h->cap_stream);
  cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
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
  CREATE_CHECK(cudaMalloc(&h->table_dev, sizeof(unsigned long long) * 42));
  CREATE_CHECK(cudaMalloc(&h->vol_dev, sizeof(VolumeArgs)));
  CREATE_CHECK(cudaMalloc(&h->rc_dev, sizeof(unsigned long long) * 2));
  CREATE_CHECK(cudaMallocHost(&h->host_pinned, 4096));

  uint64_t table[42];
  threshold_table(p, table);
  VolumeArgs va;
  std::memset(&va, 0, sizeof(va));
  va.N = h->N;
  va.epsilon = p->epsilon;
  va.cutoff2 = p->cutoff * p->cutoff;
  va.J = p->J;
  va.J_sigma = p->J_sigma;
  va.v_HB = p->v_HB;
  va.kT = p->kT;
  va.P = p->P;
  va.dV_max = p->dv_max_frac * ((double)h->N * p->v_iso_init);
  va.volume_moves = p->volume_moves;
  va.nshell = (int)d2.size();
  for (size_t i = 0; i < d2.size(); ++i) {
    va.shell_d2[i] = (double)d2[i];
    va.shell_mult[i] = (double)mult[i];
  }
  CREATE_CHECK(cudaMemcpyAsync(h->table_dev, table, sizeof(table), cudaMemcpyHostToDevice, h->stream));
  CREATE_CHECK(cudaMemcpyAsync(h->vol_dev, &va, sizeof(va), cudaMemcpyHostToDevice, h->stream));
  CREATE_CHECK(cudaMemsetAsync(h->ctrl, 0, sizeof(Ctrl), h->stream));

  h->args.state = h->state;
  h->args.ctrl = h->ctrl;
  h->args.table = h->table_dev;
  h->args.vol = h->vol_dev;
  h->args.ring = h->ring;
  h->args.ring_cap = h->ring_cap;
  h->args.keys = make_round_keys(p->seed);
  h->args.L = p->L;
  h->args.q = (uint32_t)p->q;
  h->grid_pairs = grid_for(h->N / 2, 8);
  h->grid_cells = grid_for(h->N, 8);

  k_init<<<h->grid_cells, kThreads, 0, h->stream>>>(h->state, p->L, (uint32_t)p->q,
                                                     p->init == CVF_INIT_RANDOM ? 1 : 0,
                                                     h->args.keys);
  k_set_ctrl<<<1, 32, 0, h->stream>>>(h->ctrl, (double)h->N * p->v_iso_init, 0, h->N);
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
  if (!h) return set_error(CVF_EINVAL, "handle is NULL");
  if (n_sweeps < 0 || record_every < 0)
    return set_error(CVF_EINVAL, "n_sweeps=%lld, record_every=%d must be >= 0",
                     (long long)n_sweeps, record_every);
  if (n_sweeps == 0) return CVF_OK;
  k_set_record<<<1, 32, 0, h->stream>>>(h->ctrl, record_every);
  long long left = n_sweeps;
  if (left >= kGraphSteps) {
    int rc = build_graph(h);
    if (rc) return rc;
    while (left >= h->graph_steps) {
      CVF_CUDA_CHECK(cudaGraphLaunch(h->graph, h->stream));
      left -= h->graph_steps;
    }
  }
  for (; left > 0; --left) enqueue_step(h, h->stream);
  CVF_CUDA_CHECK(cudaGetLastError());
  return CVF_OK;
}

int cvf_observables(cvf_handle* h, cvf_obs* out) {
  if (!h || !out) return set_error(CVF_EINVAL, "NULL argument");
  k_observables<<<1, 32, 0, h->stream>>>(h->vol_dev, h->ctrl, h->obs_dev);
  CVF_CUDA_CHECK(cudaGetLastError());
  CVF_CUDA_CHECK(cudaMemcpyAsync(h->host_pinned, h->obs_dev, sizeof(cvf_obs),
                                 cudaMemcpyDeviceToHost, h->stream));
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  std::memcpy(out, h->host_pinned, sizeof(cvf_obs));
  return CVF_OK;
}

int cvf_drain_series(cvf_handle* h, cvf_obs* host, int64_t cap, int64_t* n) {
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
  if (!h || !host) return set_error(CVF_EINVAL, "NULL argument");
  if ((long long)n != h->N) return set_error(CVF_EINVAL, "n=%zu, lattice has %lld cells", n, h->N);
  CVF_CUDA_CHECK(cudaMemcpyAsync(host, h->state, sizeof(uint16_t) * n, cudaMemcpyDeviceToHost,
                                 h->stream));
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  return CVF_OK;
}

int cvf_set_state(cvf_handle* h, const uint16_t* host, size_t n, double V_iso, int64_t sweep) {
  if (!h || !host) return set_error(CVF_EINVAL, "NULL argument");
  if ((long long)n != h->N) return set_error(CVF_EINVAL, "n=%zu, lattice has %lld cells", n, h->N);
  if (!(V_iso >= (double)h->N) || !std::isfinite(V_iso))
    return set_error(CVF_EINVAL, "V_iso=%g below the hard core N v0 = %lld", V_iso, h->N);
  if (sweep < 0) return set_error(CVF_EINVAL, "sweep must be >= 0");
  const uint32_t q = (uint32_t)h->p.q;
  for (size_t i = 0; i < n; ++i) {
    const uint32_t w = host[i];
    if ((w >> 12) || ((w & 7u) >= q) || (((w >> 3) & 7u) >= q) || (((w >> 6) & 7u) >= q) ||
        (((w >> 9) & 7u) >= q))
      return set_error(CVF_EINVAL, "word %zu = 0x%04x is not a valid cell for q = %u", i, w, q);
  }
  CVF_CUDA_CHECK(cudaMemcpyAsync(h->state, host, sizeof(uint16_t) * n, cudaMemcpyHostToDevice,
                                 h->stream));
  k_set_ctrl<<<1, 32, 0, h->stream>>>(h->ctrl, V_iso, sweep, h->N);
  int rc = recount_into_ctrl(h);
  if (rc) return rc;
  CVF_CUDA_CHECK(cudaStreamSynchronize(h->stream));
  h->ring_tail = 0;
  return CVF_OK;
}

int cvf_recount(cvf_handle* h, int64_t* n_hb_raw, int64_t* n_sigma) {
  if (!h || !n_hb_raw || !n_sigma) return set_error(CVF_EINVAL, "NULL argument");
  CVF_CUDA_CHECK(cudaMemsetAsync(h->rc_dev, 0, sizeof(unsigned long long) * 2, h->stream));
  k_recount<<<h->grid_cells, kThreads, 0, h->stream>>>(h->state, h->p.L, h->rc_dev);
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
  *dev_ptr = h->state;
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
