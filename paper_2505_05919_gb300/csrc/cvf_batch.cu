// cvf_batch.cu -- many independent lattices ("replicas": differing L, q, T,
// P, seeds) advanced by one persistent, cooperative, graph-captured launch:
// the host side (replica memory, launch descriptions, graphs, read-back) and
// the 256-thread kernels.  The kernel itself is in cvf_batch_kernel.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "cvf.h"
#include "cvf_batch_kernel.cuh"
#include "cvf_device.cuh"
#include "cvf_host.h"
#include "cvf_lattice.cuh"
#include "cvf_tile.cuh"

using namespace cvf;

namespace cvf {

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

}  // namespace cvf

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

// A kernel configuration: tile rows x 32-bit words (two cells per word) and
// block threads, which together fix the cells a thread updates per MC step
// (2 rows words / threads).  The first four are the automatic choices (256
// threads); the others take the same tiles with 128-thread blocks (twice the
// cells per thread) and 512-thread blocks (half), and are used when set (the
// autotuner times all).
struct TileConfig {
  int rows, words, threads, shape;  // shape: index of the tile in the kernel table
};
constexpr TileConfig kTileConfigs[] = {
    {64, 64, 256, 0}, {32, 32, 256, 1}, {32, 16, 256, 2}, {16, 16, 256, 3},
    {64, 64, 128, 0}, {32, 32, 128, 1}, {32, 16, 128, 2}, {16, 16, 128, 3},
    {64, 64, 512, 0}, {32, 32, 512, 1}, {32, 16, 512, 2}, {16, 16, 512, 3}};
constexpr int kNumTileConfigs = 12;
constexpr int kNumAutoConfigs = 4;
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

using KernelFn = BatchKernelFn;

KernelFn pick_kernel(int rng_words, bool cmp64, int cfg) {
  const TileConfig& c = kTileConfigs[cfg];
  if (c.threads == 128) return batch_kernel_nt128(rng_words, cmp64, c.shape);
  if (c.threads == 512) return batch_kernel_nt512(rng_words, cmp64, c.shape);
  return batch_kernel_for<kThreads>(rng_words, cmp64, c.shape);
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
    CVF_CUDA_CHECK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)fn,
                                                                 kTileConfigs[cfg].threads, 0));
    if (per_sm < 1) return set_error(CVF_ECUDA, "batch kernel cannot be resident");
    b->grid[cfg][c64] = per_sm * sm_count();
  }
  *grid = b->grid[cfg][c64];
  return CVF_OK;
}

// The automatic tile shape of a call: the largest whose tiles over the
// advanced replicas give every co-resident block a tile per step.  When even
// the smallest tile leaves three quarters of the blocks without one, a step
// is a latency chain through few tiles, and the same tile with 512-thread
// blocks (one cell per thread per colour) shortens each tile's part of it.
int auto_tile_config(cvf_batch* b, const std::vector<int32_t>& act, bool cmp64, int* cfg) {
  long long tiles = 0;
  int grid = 0;
  for (int c = 0; c < kNumAutoConfigs; ++c) {
    const int rc = resident_grid(b, c, cmp64, &grid);
    if (rc) return rc;
    tiles = 0;
    for (int i : act) tiles += tiles_of(b->reps[i].p.L, c);
    if (tiles >= grid) {
      *cfg = c;
      return CVF_OK;
    }
  }
  *cfg = (4 * tiles < grid) ? kNumTileConfigs - 1 : kNumAutoConfigs - 1;
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
    lc.blockDim = dim3(kTileConfigs[cfg].threads);
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

int cvf_batch_config_threads(int32_t config, int32_t* threads) {
  if (config < 0 || config >= kNumTileConfigs || !threads)
    return set_error(CVF_EINVAL, "tile config %d (0..%d)", config, kNumTileConfigs - 1);
  *threads = kTileConfigs[config].threads;
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
