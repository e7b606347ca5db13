// cvf_lattice.cuh -- launch arguments of the single-lattice kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "cvf_device.cuh"

namespace cvf {

constexpr int kThreads = 256;
// tiles of the single-lattice sweep: 64 rows x 64 words (128 cells)
constexpr int kTileRows = 64;
constexpr int kTileWords = 64;
// register budgets: five 256-thread blocks per SM (48 registers a thread;
// the most the 38 KB of shared memory of a block allows) for the
// single-lattice sweep and for the batched kernel
constexpr int kSweepBlocksPerSM = 5;
constexpr int kBatchBlocksPerSM = 5;

struct LatticeArgs {
  uint16_t* state;                   // state pair: 2 * L*L packed cell words
  Ctrl* ctrl;                        // scalar state of the lattice
  const unsigned long long* table24; // thresholds [g][(dN_HB+1)*8 + dN_sigma+3]
  const VolumeArgs* vol;             // FP64 parameters and lattice shells
  cvf_obs* ring;                     // observable ring
  long long ring_cap;
  RoundKeys keys;                    // Philox round keys of the seed
  int32_t L;
  uint32_t q;
  int32_t use_tma;                   // 1: interior tiles are staged by TMA
};

// Kernels of cvf_lattice.cu that the batch reuses for initialisation and
// observables.
__global__ void k_init(uint16_t* __restrict__ state, int32_t L, uint32_t q, int random,
                       RoundKeys K);
__global__ void k_recount(const uint16_t* __restrict__ base, int32_t L, const Ctrl* ctl,
                          unsigned long long* out);
__global__ void k_commit_counts(Ctrl* ctl);
__global__ void k_set_ctrl(const VolumeArgs* __restrict__ V, Ctrl* ctl, double V_iso,
                           long long sweep, long long N);
__global__ void k_set_record(Ctrl* ctl, int record_every);
__global__ void k_volume_prologue(const VolumeArgs* __restrict__ V, Ctrl* ctl, RoundKeys K);
__global__ void k_observables(const VolumeArgs* __restrict__ V, const Ctrl* ctl,
                              const unsigned long long* hist, cvf_obs* out);
__global__ void k_histogram(const uint16_t* __restrict__ state, long long N,
                            unsigned long long* out);

// The resident sweep (cvf_resident2.cu): a square lattice of side L (a
// multiple of kResCtas, 2 kResCtas <= L <= kResMaxSide) held in the shared
// memory of one cluster of kResCtas CTAs for many steps per launch.
constexpr int kResCtas = 8;
constexpr int kResMaxSide = 256;
bool resident_fits(const LatticeArgs& A, int rng_words, bool cmp64);
cudaError_t launch_resident(const LatticeArgs& A, int rng_words, bool cmp64, long long n_steps,
                            cudaStream_t s);

// Host helpers shared by both paths.
void fill_volume_args(const cvf_params* p, long long N, const std::vector<int64_t>& d2,
                      const std::vector<int64_t>& mult, VolumeArgs* va);
bool fill_table24(const cvf_params* p, unsigned long long table24[48]);

}  // namespace cvf
