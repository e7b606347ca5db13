// cvf_resident2.cu -- the checkerboard sweep of a small square lattice kept
// resident in the shared memory of one thread-block cluster for many MC
// steps per launch.
//
// The cluster's kResCtas CTAs each hold L / kResCtas consecutive rows.  A
// step is: colour 0 over every CTA's rows, a cluster barrier, colour 1 with
// the counts of the step gathered into CTA 0 through distributed shared
// memory, a cluster barrier, CTA 0 committing the step (finalize_step:
// counts, ring record, volume move), and a last barrier.  The rows just above and below a
// CTA's slab are read from the neighbouring CTAs' shared memory.  Each cell
// is updated exactly as in the tiled sweep (update_in_word: the same draws,
// the same rule), so the lattice and every count are those of the tiled path.
// Two extra warps of CTA 0 decide the next step's volume move while the
// colours run (it needs no bonds unless the gate would change), each on its
// own FP64 pipe (volume_decide_pair).
//
// Every CTA runs the same loop of steps with the same barriers; no CTA leaves
// early, so the hardware barriers always complete.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

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

// Cluster barrier in two halves (PTX barrier.cluster: arrive releases, wait
// acquires): a thread may work between its arrival and its wait.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait;" ::: "memory"); }
__device__ __forceinline__ void cluster_barrier() {
  cluster_arrive();
  cluster_wait();
}

// Barrier of the sweeping threads of a CTA only (named barrier 1), so that
// the volume warp never holds them up.
__device__ __forceinline__ void sweepers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(kResThreads) : "memory");
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
  const int nctas = (int)cluster.num_blocks();
  extern __shared__ uint32_t lat[];  // rows y0 .. y0 + R - 1 of the lattice, Lh words each
  __shared__ Tables2 Tb;
  __shared__ unsigned long long s_acc[3];   // CTA 0: the step's dN_HB, dN_sigma, moves
  __shared__ unsigned long long s_hist[8];  // CTA 0: N_q' of a recorded step
  __shared__ uint32_t s_hist4[4];
  __shared__ int s_next_g;                  // CTA 0: the gate of the next step
  __shared__ VolumeArgs sV;                 // FP64 parameters for the volume moves
  __shared__ double s_xch;                  // the two volume warps' exchange
  // CTA 0 keeps the lattice's scalar state in shared memory for the whole
  // call (no other launch touches it meanwhile) and writes it back at the
  // end, so no step waits on a global-memory round trip
  __shared__ Ctrl s_ctl;
  Ctrl* const gctl = A.ctrl;
  const int L = A.L, Lh = L >> 1, R = L / nctas, y0 = rank * R;
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
  const uint32_t* up = cluster.map_shared_rank(lat, (rank + nctas - 1) % nctas) + (R - 1) * Lh;
  const uint32_t* down = cluster.map_shared_rank(lat, (rank + 1) % nctas);
  unsigned long long* acc0 = cluster.map_shared_rank(&s_acc[0], 0);
  unsigned long long* hist0 = cluster.map_shared_rank(&s_hist[0], 0);
  const int* next_g0 = cluster.map_shared_rank(&s_next_g, 0);
  int g_cur = -1;
  __syncthreads();
  cluster_barrier();

  // Three cluster barriers per step: (1) colour 0 done, (2) colour 1 and the
  // counts done, (3) the step committed by CTA 0.  The volume warp arrives
  // at (1) at once and decides the next step's move before it waits, so its
  // FP64 work overlaps both colours.
  for (long long it = 0; it < n_steps; ++it) {
    const long long step = step0 + it;
    const bool rec = step_recorded(every, step);
    if (!sweeper) {
      cluster_arrive();  // (1)
      if (rank == 0) {  // the two volume warps: the move on two FP64 pipes
        VolumeResult r;
        const bool ok = volume_decide_pair<3>((int)((threadIdx.x - kResThreads) >> 5), sV,
                                              step + 1, ctl->next_V, ctl->next_u, ctl->next_g,
                                              -1, K, &r, &s_xch);
        if (threadIdx.x == kResThreads && ok) {
          ctl->ahead_V = r.V;
          ctl->ahead_u = r.u;
          ctl->ahead_g = r.g;
          ctl->ahead_acc = r.accepted;
          ctl->ahead_state = 1;
        }
      }
      __syncwarp();
      cluster_wait();     // (1)
      cluster_barrier();  // (2)
      cluster_barrier();  // (3)
      continue;
    }
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
                                                  KeysRound{&K}, A.q, Tb, pk,
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
  const size_t smem = (size_t)(L / kResCtas) * (L / 2) * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(kResCtas);
  cfg.blockDim = dim3(kResBlock);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = kResCtas;
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
