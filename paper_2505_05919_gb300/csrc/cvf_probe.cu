// cvf_probe.cu -- measurement and failure-detection aids beside the sweep:
// the byte-roofline probe (a plain 16-byte vector copy whose event-timed
// bandwidth on a given working set -- two buffers that fit in L2, or two much
// larger than L2 -- is the denominator for the sweep's algorithmic bytes,
// read 2 B + write 2 B per cell and step), the random-number ceiling (one
// Philox4x32-10 block per cell and nothing else: the draws a sweep must
// make), and the bounded device wait of the persistent batched sweep run
// alone on a flag, so that its give-up path is exercised without a fault.
#include <cuda_runtime.h>

#include <cstdint>

#include "cvf_device.cuh"
#include "cvf_host.h"

namespace cvf {
namespace {

constexpr int kCopyThreads = 256;
constexpr int kCopyUnroll = 4;

// Every thread moves kCopyUnroll vectors per iteration: all loads are issued
// before the first store, so each thread keeps 64 bytes in flight.
__global__ void __launch_bounds__(kCopyThreads) k_copy16(const uint4* __restrict__ src,
                                                          uint4* __restrict__ dst, size_t n) {
  const size_t stride = (size_t)gridDim.x * kCopyThreads;
  size_t i = (size_t)blockIdx.x * kCopyThreads + threadIdx.x;
  for (; i + (kCopyUnroll - 1) * stride < n; i += kCopyUnroll * stride) {
    uint4 v[kCopyUnroll];
#pragma unroll
    for (int u = 0; u < kCopyUnroll; ++u) v[u] = src[i + u * stride];
#pragma unroll
    for (int u = 0; u < kCopyUnroll; ++u) dst[i + u * stride] = v[u];
  }
  for (; i < n; i += stride) dst[i] = src[i];
}

// The random-number ceiling of a sweep: every cell c < n draws the one
// Philox4x32-10 block a checkerboard step must draw for it, counter (c,
// step, tag 0), key = the seed, with the same device function the sweep
// kernels call, and nothing else; the four words of every block are
// XOR-folded so that no draw can be removed, and each warp adds its fold to
// *out with one atomic XOR.  Its event-timed rate, four sigma updates per
// cell, is the most a sweep that draws its numbers this way can reach.
__global__ void __launch_bounds__(kCopyThreads) k_philox_probe(uint32_t n, uint32_t step_lo,
                                                               uint32_t step_hi, RoundKeys K,
                                                               unsigned int* out) {
  uint32_t fold = 0;
  const uint32_t stride = gridDim.x * kCopyThreads;
  for (uint32_t c = blockIdx.x * kCopyThreads + threadIdx.x; c < n; c += stride) {
    const Words4 r = philox(c, step_lo, step_hi, kTagAccept, K);
    fold ^= (r.x ^ r.y) ^ (r.z ^ r.w);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fold ^= __shfl_xor_sync(0xFFFFFFFFu, fold, o);
  if ((threadIdx.x & 31u) == 0u && fold) atomicXor(out, fold);
}

// One thread waits for *flag >= target exactly as a batched tile waits for
// its replica; the outcome (WaitResult) goes to *result.
__global__ void k_wait_probe(const unsigned int* flag, unsigned int target, unsigned int limit,
                             unsigned int* result) {
  if (blockIdx.x == 0 && threadIdx.x == 0)
    *result = (unsigned int)wait_flag_geq(flag, target, nullptr, limit);
}

}  // namespace
}  // namespace cvf

using namespace cvf;

extern "C" int cvf_wait_probe(const uint32_t* flag, uint32_t target, uint32_t polls, void* stream) {
  clear_error();
  if (!flag) return set_error(CVF_EINVAL, "cvf_wait_probe: NULL flag");
  if (reinterpret_cast<uintptr_t>(flag) & 3u)
    return set_error(CVF_EINVAL, "cvf_wait_probe: flag must be 4-byte aligned");
  if (polls < 1 || polls > kWaitPollLimit)
    return set_error(CVF_EINVAL, "cvf_wait_probe: polls=%u outside 1..%u", polls, kWaitPollLimit);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  unsigned int* d_result = nullptr;
  CVF_CUDA_CHECK(cudaMalloc(&d_result, sizeof(unsigned int)));
  unsigned int h_result = 0xFFFFFFFFu;
  cudaError_t e = cudaMemsetAsync(d_result, 0xFF, sizeof(unsigned int), s);
  if (e == cudaSuccess) {
    k_wait_probe<<<1, 32, 0, s>>>(reinterpret_cast<const unsigned int*>(flag), target, polls,
                                  d_result);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h_result, d_result, sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_result);
  if (e != cudaSuccess)
    return set_error(CVF_ECUDA, "cvf_wait_probe: %s", cudaGetErrorString(e));
  if (h_result == (unsigned int)kWaitGaveUp)
    return set_error(CVF_ETIMEOUT, "cvf_wait_probe: the flag did not reach %u within %u polls",
                     target, polls);
  if (h_result != (unsigned int)kWaitDone)
    return set_error(CVF_ECUDA, "cvf_wait_probe: unexpected wait result %u", h_result);
  return CVF_OK;
}

extern "C" int cvf_copy_probe(void* dst, const void* src, size_t bytes, void* stream) {
  clear_error();
  if (!dst || !src) return set_error(CVF_EINVAL, "cvf_copy_probe: NULL buffer");
  if ((bytes & 15u) || (reinterpret_cast<uintptr_t>(dst) & 15u) ||
      (reinterpret_cast<uintptr_t>(src) & 15u))
    return set_error(CVF_EINVAL, "cvf_copy_probe: buffers and size must be 16-byte aligned");
  if (bytes == 0) return CVF_OK;
  const size_t n = bytes / 16u;
  // eight resident blocks of 256 threads per SM fill every SM
  const size_t want = (n + kCopyThreads - 1) / kCopyThreads;
  const size_t cap = (size_t)sm_count() * 8u;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  k_copy16<<<grid, kCopyThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const uint4*>(src), reinterpret_cast<uint4*>(dst), n);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_error(CVF_ECUDA, "cvf_copy_probe: launch failed: %s", cudaGetErrorString(e));
  return CVF_OK;
}

extern "C" int cvf_philox_probe(uint64_t seed, uint32_t n_cells, int64_t step, uint32_t* dev_out,
                                void* stream) {
  clear_error();
  if (!dev_out) return set_error(CVF_EINVAL, "cvf_philox_probe: NULL output word");
  if (reinterpret_cast<uintptr_t>(dev_out) & 3u)
    return set_error(CVF_EINVAL, "cvf_philox_probe: output word must be 4-byte aligned");
  if (step < 0) return set_error(CVF_EINVAL, "cvf_philox_probe: step must be >= 0");
  if (n_cells == 0) return CVF_OK;
  // as many 256-thread blocks as are resident at once (8 per SM), each
  // thread taking cells a grid apart
  const size_t want = ((size_t)n_cells + kCopyThreads - 1) / kCopyThreads;
  const size_t cap = (size_t)sm_count() * 8u;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  k_philox_probe<<<grid, kCopyThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      n_cells, (uint32_t)((uint64_t)step & 0xFFFFFFFFu), (uint32_t)((uint64_t)step >> 32),
      make_round_keys(seed), reinterpret_cast<unsigned int*>(dev_out));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return set_error(CVF_ECUDA, "cvf_philox_probe: launch failed: %s", cudaGetErrorString(e));
  return CVF_OK;
}
