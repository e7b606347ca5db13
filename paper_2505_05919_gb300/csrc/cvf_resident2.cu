// cvf_resident2.cu -- the checkerboard sweep of a small square lattice kept
// resident in the shared memory of one thread-block cluster for many MC
// steps per launch.
//
// The cluster's first kResCtas CTAs each hold L / kResCtas consecutive rows.  A
// step is: colour 0 over every CTA's rows, a cluster barrier, colour 1 with
// the counts of the step gathered into CTA 0 through distributed shared
// memory, a cluster barrier, CTA 0 committing the step (finalize_step:
// counts, ring record, volume move), and a last barrier.  The rows just above and below a
// CTA's slab are read from the neighbouring CTAs' shared memory.  Each cell
// is updated exactly as in the tiled sweep (update_in_word: the same draws,
// the same rule), so the lattice and every count are those of the tiled path.
// Two warps of one more CTA decide the coming steps' volume moves ahead while
// the colours and the commit run (they need no bonds unless the gate would
// change), in passes over a tree of outcomes (the volume engine below).
//
// Every CTA runs the same loop of steps with the same barriers; no CTA leaves
// early, so the hardware barriers always complete.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "cvf_device.cuh"
#include "cvf_host.h"
#include "cvf_lattice.cuh"
#include "cvf_tile.cuh"

namespace cg = cooperative_groups;

namespace cvf {
namespace {

constexpr int kResThreads = 256;            // sweeping threads per CTA
constexpr int kResBlock = kResThreads + 64;  // + two volume warps
// The cluster: kResCtas CTAs hold the lattice, one more (rank kResCtas)
// runs the volume engine.  On GB300 an FP64 instruction holds back the
// integer multiply-adds of the warps that share its SM sub-partition, so
// the engine gets an SM of its own: every CTA asks for at least
// kResMinSmem bytes of shared memory, which lets only one CTA of the
// cluster on an SM.
constexpr int kResCluster = kResCtas + 1;
constexpr size_t kResMinSmem = 120 * 1024;

// Cluster barrier in two halves (PTX barrier.cluster: arrive releases, wait
// acquires): a thread may work between its arrival and its wait.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait;" ::: "memory"); }
__device__ __forceinline__ void cluster_barrier() {
  cluster_arrive();
  cluster_wait();
}

// Barrier of the sweeping threads of a CTA only (named barrier 1), so that
// the volume warps never hold them up.
__device__ __forceinline__ void sweepers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kResThreads) : "memory");
}

// ---------------------------------------------------------------------------
// The volume chain run ahead.  While no proposal would change the gate, the
// volume moves of the coming steps do not depend on the bonds: the move of
// step s+1 follows from the state after step s's move and the step's two
// draws alone (Sec. II.B step 1).  The two volume warps of the engine CTA
// decide them ahead, kEngDepth steps per pass, over the tree of outcomes:
// node i (heap order, lane i) is the move of step t0 + depth(i) from the
// state that the accept / reject outcomes on its path lead to.  An FP64
// instruction holds the pipe for a whole warp whatever the number of active
// lanes, so a pass over 31 lanes costs about what one decision costs, and
// the walk from the root along the computed outcomes settles up to five
// steps.  Each node runs the IEEE operations of volume_decide_pair in the
// same order, so every move equals the step-by-step chain's.  A node whose
// proposal would change the gate needs the bonds of the step before it: the
// walk stops there, the commit of that step decides it (finalize_step), and
// the engine restarts from the committed state.  A pass is cut into
// kEngStages stages, one per barrier segment of the step (three per step),
// so that no stage holds up the sweep for long; decided moves wait in a ring
// and reach the commit through CTA 0's ctl->ahead_* (distributed shared
// memory, published before the step's commit).
constexpr int kEngDepth = 5;   // steps per pass: 31 nodes
constexpr int kEngStages = 10;
constexpr int kEngRing = 16;   // decided moves kept (steps step+1 .. step+9 at most)
// A pass starts while the moves known reach at most kEngLead steps past the
// current one: its kEngStages stages end about 3.3 steps later, a step
// before its first move is needed.
constexpr int kEngLead = 4;
constexpr int kEngBar = 4;     // named barrier of the two volume warps

struct EngineMove {
  double V, u;
  int g, acc;
};

struct EngineCtl {
  long long dec_hi;   // last step whose move is known (committed or in the ring)
  long long blocked;  // step whose proposal would change the gate (its commit decides it), or -1
  long long t0;       // root step of the pass in flight
  long long published;  // last step whose move went to ctl->ahead_*
  double bV, bu;      // the state after the move of step dec_hi
  int bg;
  int stage;          // next stage of the pass in flight, -1: none
};

// A lane's values of the pass in flight (registers of the volume warps).
struct EngineLane {
  double dV, u2, Vo, Vn, vn, ratio, x, un, dH, q;
  int k, g_new;
  bool hard, met;  // hard core (v' < 1); the Metropolis test passed
};

__device__ __forceinline__ void engine_pair_sync() {
  asm volatile("bar.sync %0, 64;" ::"n"(kEngBar) : "memory");
}

// One stage of the pass rooted at c.t0 from the state (c.bV, c.bu, c.bg).
// Role 0 evaluates the energy change, role 1 the log of the volume ratio
// (into xch[lane]).  Stage kEngStages - 1 walks the tree, fills the ring and
// updates c (every lane alike).
__device__ __forceinline__ void engine_stage(int role, EngineCtl& c, EngineLane& e,
                                             EngineMove* ring, double* xch,
                                             const VolumeArgs& V, const RoundKeys& K) {
  const unsigned int full = 0xFFFFFFFFu;
  const int lane = (int)(threadIdx.x & 31u);
  const int n1 = lane + 1;            // 1-based heap index: children 2 n1 (reject), 2 n1 + 1 (accept)
  const int d = 31 - __clz(n1);       // depth: the node is the move of step t0 + d
  const double Nd = (double)V.N;
  switch (c.stage) {
    case 0: {
      const long long st = c.t0 + d;
      const Words4 r = philox(kCellVolume, (uint32_t)((unsigned long long)st & 0xFFFFFFFFu),
                              (uint32_t)((unsigned long long)st >> 32), kTagVolume, K);
      const double u1 = u53(r.x, r.y);
      e.u2 = u53(r.z, r.w);
      e.dV = (2.0 * u1 - 1.0) * V.dV_max;
      break;
    }
    case 1: {
      // the volume before the node's move: the accepted moves on its path,
      // added in step order (lane 2^j - 1 holds the draw of depth j)
      double Vo = c.bV;
#pragma unroll
      for (int j = 0; j < kEngDepth; ++j) {
        const double dVj = __shfl_sync(full, e.dV, (1 << j) - 1);
        if (j < d && ((n1 >> (d - 1 - j)) & 1)) Vo = Vo + dVj;
      }
      e.Vo = Vo;
      e.Vn = Vo + e.dV;
      break;
    }
    case 2:
      if (role == 0)
        e.vn = e.Vn / Nd;
      else
        e.ratio = e.Vn / e.Vo;
      break;
    case 3:
      if (role == 0) {
        e.hard = e.vn < 1.0;
        e.g_new = (e.vn < 2.0) ? 1 : 0;
        e.k = lj_shells_inside(V, e.vn);
      } else {
        xch[lane] = Nd * log(e.ratio);
      }
      break;
    case 4:
      if (role == 0) e.x = 1.0 / e.vn;
      break;
    case 5:
      if (role == 0) {
        const double x3 = e.x * e.x * e.x;
        const double x6 = x3 * x3;
        e.un = (2.0 * V.epsilon) * (x6 * V.S12[e.k] - x3 * V.S6[e.k]);
      }
      break;
    case 6:
      if (role == 0) {
        // the energy before the move: that of the last accepted move on the
        // path (its lane), else the pass's starting state's
        int src = -1;
#pragma unroll
        for (int j = 0; j < kEngDepth; ++j)
          if (j < d && ((n1 >> (d - 1 - j)) & 1)) src = (n1 >> (d - j)) - 1;
        const double uo_lane = __shfl_sync(full, e.un, src < 0 ? lane : src);
        const double uo = (src < 0) ? c.bu : uo_lane;
        const double J_eff = V.J - V.P * V.v_HB;
        const double du = e.un - uo;
        const double t1 = Nd * du;
        const double t2 = V.P * e.dV;
        const double t3 = ((double)(e.g_new - c.bg) * J_eff) * (double)0;
        e.dH = (t1 + t2) - t3;
      }
      break;
    case 7:
      if (role == 0) e.q = -e.dH / V.kT;
      break;
    case 8:
      if (role == 0) {
        const double arg = e.q + xch[lane];
        e.met = e.u2 < exp(arg);
      }
      break;
    case kEngStages - 1: {
      // walk the tree along the outcomes; every lane takes the same path
      const bool node = lane < 31;
      const bool flip = !e.hard && e.g_new != c.bg;
      const bool acc = !e.hard && !flip && e.met;
      const unsigned int A = __ballot_sync(full, node && acc && role == 0);
      const unsigned int U = __ballot_sync(full, node && flip && role == 0);
      double Vc = c.bV, uc = c.bu;
      int nn = 1, j = 0;
      for (; j < kEngDepth; ++j) {
        const int i = nn - 1;
        if ((U >> i) & 1u) break;
        const int a = (int)((A >> i) & 1u);
        const double Vi = __shfl_sync(full, e.Vn, i);
        const double ui = __shfl_sync(full, e.un, i);
        if (a) {
          Vc = Vi;
          uc = ui;
        }
        if (role == 0 && lane == 0) {
          EngineMove& m = ring[(c.t0 + j) & (kEngRing - 1)];
          m.V = Vc;
          m.u = uc;
          m.g = c.bg;
          m.acc = a;
        }
        nn = 2 * nn + a;
      }
      c.dec_hi = c.t0 + j - 1;
      if (j < kEngDepth) c.blocked = c.t0 + j;
      c.bV = Vc;
      c.bu = uc;
      c.stage = -1;
      return;
    }
    default:
      break;
  }
  ++c.stage;
}

// One barrier segment of the engine, run by both volume warps of CTA 0.
// `first`: the segment after the step's first arrival, where the committed
// move of `step` (finalize_step of the step before) can be read.  The move
// of step + 1 is published for the step's commit as soon as it is known
// (in a segment that ends before the commit starts: `may_publish`).
// The control state is double-buffered by segment parity (cs[par] is read,
// cs[par ^ 1] written), so one barrier of the two warps per segment orders
// every read before the next write of the same buffer.
__device__ __forceinline__ void engine_segment(bool first, bool may_publish, long long step,
                                               int par, int role, EngineCtl* cs, EngineLane& e,
                                               EngineMove* ring, double* xch, Ctrl* ctl,
                                               const VolumeArgs& V, const RoundKeys& K) {
  engine_pair_sync();  // the other warp's writes of the last segment are visible
  EngineCtl c = cs[par];
  if (first) {
    // the engine stopped at a gate change that a commit has decided since,
    // or fell behind with no pass in flight: restart from the committed move
    if ((c.blocked >= 0 && c.blocked <= step) || (c.stage < 0 && c.dec_hi < step)) {
      c.dec_hi = step;
      c.blocked = -1;
      c.stage = -1;
      c.bV = ctl->next_V;
      c.bu = ctl->next_u;
      c.bg = ctl->next_g;
    }
  }
  if (c.stage < 0 && c.blocked < 0 && c.dec_hi <= step + kEngLead) {
    c.stage = 0;
    c.t0 = c.dec_hi + 1;
  }
  if (c.stage >= 0) engine_stage(role, c, e, ring, xch, V, K);
  if (may_publish && c.published < step + 1 && c.dec_hi >= step + 1) {
    if (role == 0 && (threadIdx.x & 31u) == 0) {
      const EngineMove m = ring[(step + 1) & (kEngRing - 1)];
      ctl->ahead_V = m.V;
      ctl->ahead_u = m.u;
      ctl->ahead_g = m.g;
      ctl->ahead_acc = m.acc;
      ctl->ahead_state = 1;
    }
    c.published = step + 1;
  }
  if (role == 0 && (threadIdx.x & 31u) == 0) cs[par ^ 1] = c;
}

// Sum of three counters over the sweeping threads; valid in thread 0.
__device__ __forceinline__ void sweepers_sum3(uint32_t& a, uint32_t& b, uint32_t& c) {
  __shared__ uint32_t red[3][kResThreads / 32];
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
  sweepers_sync();
  if (threadIdx.x == 0) {
    a = 0;
    b = 0;
    c = 0;
#pragma unroll
    for (int i = 0; i < kResThreads / 32; ++i) {
      a += red[0][i];
      b += red[1][i];
      c += red[2][i];
    }
  }
}

template <int RNG_WORDS, bool CMP64>
__global__ void __launch_bounds__(kResBlock) k_resident2(LatticeArgs A, long long n_steps) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int nctas = kResCtas;                 // the CTAs that hold rows
  const bool engine_cta = rank == kResCtas;   // the volume engine's CTA
  extern __shared__ uint32_t lat[];  // rows y0 .. y0 + R - 1 of the lattice, Lh words each
  __shared__ Tables2 Tb;
  __shared__ unsigned long long s_acc[3];   // CTA 0: the step's dN_HB, dN_sigma, moves
  __shared__ unsigned long long s_hist[8];  // CTA 0: N_q' of a recorded step
  __shared__ uint32_t s_hist4[4];
  __shared__ int s_next_g;                  // CTA 0: the gate of the next step
  __shared__ VolumeArgs sV;                 // FP64 parameters for the volume moves
  __shared__ EngineCtl s_eng[2];            // engine CTA: the volume chain run ahead
  __shared__ EngineMove s_ring[kEngRing];
  __shared__ double s_lr[32];               // the log warp's values, per node
  // CTA 0 keeps the lattice's scalar state in shared memory for the whole
  // call (no other launch touches it meanwhile) and writes it back at the
  // end, so no step waits on a global-memory round trip
  __shared__ Ctrl s_ctl;
  Ctrl* const gctl = A.ctrl;
  const int L = A.L, Lh = L >> 1, R = engine_cta ? 0 : L / nctas, y0 = engine_cta ? 0 : rank * R;
  const long long N = (long long)L * L;
  const bool sweeper = threadIdx.x < kResThreads;
  const long long step0 = gctl->sweep;
  const int every = gctl->record_every;
  if (rank == 0 && threadIdx.x == 0) s_ctl = *gctl;
  Ctrl* const ctl = &s_ctl;  // meaningful in CTA 0 only
  const RoundKeys& K = A.keys;

  // own rows from the source buffer of the first step
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(A.state + (size_t)(step0 & 1) * N);
    for (int i = threadIdx.x; i < R * Lh; i += blockDim.x) lat[i] = src[(size_t)y0 * Lh + i];
  }
  fill_prop2(Tb, A.q);
  stage_volume_args(&sV, A.vol);
  if (rank == 0 && threadIdx.x == 0) s_next_g = ctl->next_g;
  if (threadIdx.x < 4) s_hist4[threadIdx.x] = 0;
  // the rows of the CTAs above and below (periodic), in their shared memory
  // (the engine CTA holds no rows and reads none)
  const int nb_up = engine_cta ? 0 : (rank + nctas - 1) % nctas;
  const int nb_down = engine_cta ? 0 : (rank + 1) % nctas;
  const uint32_t* up = cluster.map_shared_rank(lat, nb_up) + (L / nctas - 1) * Lh;
  const uint32_t* down = cluster.map_shared_rank(lat, nb_down);
  unsigned long long* acc0 = cluster.map_shared_rank(&s_acc[0], 0);
  unsigned long long* hist0 = cluster.map_shared_rank(&s_hist[0], 0);
  const int* next_g0 = cluster.map_shared_rank(&s_next_g, 0);
  Ctrl* const ctl0 = cluster.map_shared_rank(&s_ctl, 0);  // CTA 0's scalar state
  int g_cur = -1;
  __syncthreads();
  cluster_barrier();
  if (engine_cta && threadIdx.x == kResThreads) {
    // the move of step0 is committed; the engine starts from it
    EngineCtl& c = s_eng[0];
    c.dec_hi = step0;
    c.blocked = -1;
    c.t0 = step0 + 1;
    c.published = step0;
    c.bV = ctl0->next_V;
    c.bu = ctl0->next_u;
    c.bg = ctl0->next_g;
    c.stage = -1;
  }

  // Three cluster barriers per step: (1) colour 0 done, (2) colour 1 and the
  // counts done, (3) the step committed by CTA 0.  The volume warps arrive
  // at each barrier as soon as they reach it and run one stage of the
  // volume engine before they wait, so their FP64 work overlaps colour 0,
  // colour 1 and the commit in turn.
  if (!sweeper) {
    const bool engine = engine_cta && sV.volume_moves != 0;
    const int role = (int)((threadIdx.x - kResThreads) >> 5);
    EngineLane e;
    e.hard = false;
    e.met = false;
    for (long long it = 0; it < n_steps; ++it) {
      const long long step = step0 + it;
      // three segments per step: parities 0 1 0, 1 0 1, ... by 3 it + k
      const int par = (int)((3 * it) & 1);
      cluster_arrive();  // (1)
      if (engine)
        engine_segment(true, true, step, par, role, s_eng, e, s_ring, s_lr, ctl0, sV, K);
      __syncwarp();
      cluster_wait();
      cluster_arrive();  // (2)
      if (engine)
        engine_segment(false, true, step, par ^ 1, role, s_eng, e, s_ring, s_lr, ctl0, sV, K);
      __syncwarp();
      cluster_wait();
      cluster_arrive();  // (3): the commit runs meanwhile
      if (engine)
        engine_segment(false, false, step, par, role, s_eng, e, s_ring, s_lr, ctl0, sV, K);
      __syncwarp();
      cluster_wait();
    }
  }
  // the engine CTA's other warps hold no rows: they only keep the barriers
  for (long long it = 0; sweeper && engine_cta && it < n_steps; ++it) {
    cluster_barrier();  // (1)
    cluster_barrier();  // (2)
    cluster_barrier();  // (3)
  }
  for (long long it = 0; sweeper && !engine_cta && it < n_steps; ++it) {
    const long long step = step0 + it;
    const bool rec = step_recorded(every, step);
    const int g = *next_g0;
    if (g != g_cur) {  // uniform over the CTA's sweepers
      fill_rows2(Tb, A.table24, g);
      g_cur = g;
    }
    if (rank == 0 && threadIdx.x < 3) s_acc[threadIdx.x] = 0;
    if (rank == 0 && threadIdx.x < 8) s_hist[threadIdx.x] = 0;
    sweepers_sync();
    const uint32_t s_lo = (uint32_t)((unsigned long long)step & 0xFFFFFFFFu);
    const uint32_t s_hi = (uint32_t)((unsigned long long)step >> 32);
    TileCounts cnt{0, 0, 0};
    for (int colour = 0; colour < 2; ++colour) {
      uint32_t pk = 0;
      for (int i = threadIdx.x; i < R * Lh; i += kResThreads) {
        const int r = i / Lh, p = i - r * Lh;
        if (!dcheck(r >= 0 && r < R && p >= 0 && p < Lh, &gctl->error, kSiteResident2)) continue;
        const int y = y0 + r;
        const int hi = (y & 1) ^ colour;  // the cell of this colour in word (y, p)
        const uint32_t own = lat[i];
        const uint32_t xm = lat[r * Lh + (p == 0 ? Lh - 1 : p - 1)];
        const uint32_t xp = lat[r * Lh + (p + 1 == Lh ? 0 : p + 1)];
        const uint32_t ym = (r == 0) ? up[p] : lat[i - Lh];
        const uint32_t yp = (r == R - 1) ? down[p] : lat[i + Lh];
        lat[i] = update_in_word<RNG_WORDS, CMP64>(own, xm, xp, ym, yp, hi,
                                                  (uint32_t)(y * L + 2 * p + hi), s_lo, s_hi,
                                                  KeysInRegs{A.keys}, A.q, Tb, pk,
                                                  rec ? s_hist4 : nullptr);
      }
      cnt.add(pk);
      if (colour == 0) cluster_barrier();  // (1)
    }
    // the step's counts (and N_q') into CTA 0
    uint32_t dhb = (uint32_t)cnt.dhb(), dc = (uint32_t)cnt.dc(), nacc = cnt.nacc;
    sweepers_sum3(dhb, dc, nacc);
    if (threadIdx.x == 0) {
      atomicAdd(&acc0[0], (unsigned long long)(long long)(int)dhb);
      atomicAdd(&acc0[1], (unsigned long long)(long long)(int)dc);
      atomicAdd(&acc0[2], (unsigned long long)nacc);
    }
    if (rec) {
      sweepers_sync();
      if (threadIdx.x < 4) {
        const uint32_t w = s_hist4[threadIdx.x];
        if (w & 0xFFFFu) atomicAdd(&hist0[threadIdx.x], (unsigned long long)(w & 0xFFFFu));
        if (w >> 16) atomicAdd(&hist0[threadIdx.x + 4], (unsigned long long)(w >> 16));
        s_hist4[threadIdx.x] = 0;
      }
    }
    cluster_barrier();  // (2)
    if (rank == 0 && threadIdx.x == 0) {
      ctl->acc_hb = s_acc[0];
      ctl->acc_pairs = s_acc[1];
      ctl->acc_moves = s_acc[2];
      if (rec)
        for (int v = 0; v < 8; ++v) ctl->acc_hist[v] = s_hist[v];
      finalize_step<true>(sV, ctl, A.ring, A.ring_cap, K);
      s_next_g = ctl->next_g;
    }
    cluster_barrier();  // (3)
  }

  // CTA 0's scalar state back to the handle (every CTA is past its last
  // index check, so the device error word is final)
  if (rank == 0 && threadIdx.x == 0) {
    s_ctl.error = *(volatile unsigned int*)&gctl->error;
    *gctl = s_ctl;
  }
  // own rows to the buffer that holds the lattice after the last step
  __syncthreads();
  uint32_t* dst = reinterpret_cast<uint32_t*>(A.state + (size_t)((step0 + n_steps) & 1) * N);
  for (int i = threadIdx.x; i < R * Lh; i += blockDim.x) dst[(size_t)y0 * Lh + i] = lat[i];
}

template <int RNG_WORDS, bool CMP64>
cudaError_t launch_t(const LatticeArgs& A, long long n_steps, cudaStream_t s, bool query,
                     int* clusters) {
  const void* fn = (const void*)k_resident2<RNG_WORDS, CMP64>;
  const int L = A.L;
  const size_t smem =
      std::max((size_t)(L / kResCtas) * (L / 2) * sizeof(uint32_t), kResMinSmem);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(kResCluster);
  cfg.blockDim = dim3(kResBlock);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kResCluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (query) return cudaOccupancyMaxActiveClusters(clusters, fn, &cfg);
  return cudaLaunchKernelEx(&cfg, k_resident2<RNG_WORDS, CMP64>, A, n_steps);
}

cudaError_t dispatch(const LatticeArgs& A, int rng_words, bool cmp64, long long n_steps,
                     cudaStream_t s, bool query, int* clusters) {
  if (rng_words == 1)
    return cmp64 ? launch_t<1, true>(A, n_steps, s, query, clusters)
                 : launch_t<1, false>(A, n_steps, s, query, clusters);
  return cmp64 ? launch_t<2, true>(A, n_steps, s, query, clusters)
               : launch_t<2, false>(A, n_steps, s, query, clusters);
}

}  // namespace

bool resident_fits(const LatticeArgs& A, int rng_words, bool cmp64) {
  const int L = A.L;
  if (L < 2 * kResCtas || L > kResMaxSide || L % kResCtas != 0) return false;
  int clusters = 0;
  if (dispatch(A, rng_words, cmp64, 0, nullptr, true, &clusters) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return clusters >= 1;
}

cudaError_t launch_resident(const LatticeArgs& A, int rng_words, bool cmp64, long long n_steps,
                            cudaStream_t s) {
  return dispatch(A, rng_words, cmp64, n_steps, s, false, nullptr);
}

}  // namespace cvf
