// cvf_lattice.cuh -- launch arguments of the single-lattice kernels.
#pragma once
#include <cuda.h>  // CUtensorMap
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
// the most the 40 KB of shared memory of a 64 x 64-word tile allows) for the
// single-lattice tiled sweep; four (64 registers) for the batched kernel,
// which keeps its item's replica state across the colour phases (the 256
// replicas of the batched workload: 140.8 against 148.3 us per step on the
// 64 x 64-word tiles the autotuner picks)
constexpr int kSweepBlocksPerSM = 5;
constexpr int kBatchBlocksPerSM = 4;
// the wavefront sweep keeps more state across its items (the item, its
// dependencies, the counts not yet reported): four blocks per SM at 64
// registers (at five blocks, 48 registers, its column-walking form spills
// about 220 bytes and runs 6 % slower at 4096^2: 115.9 against 108.6 us per
// step)
constexpr int kWaveBlocksPerSM = 4;

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

// The wavefront sweep (cvf_wave.cu): one persistent cooperative launch per
// call, a tile of step s + 1 waiting only for the 3 x 3 tiles around it to
// finish step s, the volume moves decided ahead by block 0.  Its scratch in
// device memory: this header, then one progress word per tile.
constexpr int kWaveRing = 16;  // MC steps in flight at most
struct WaveMove {              // the volume move of a step, published by the engine
  double V, u;
  int g, acc;
  unsigned int tag;            // relative step + 1 once published
  unsigned int pad;
};
struct WaveAcc {               // a step's counts, added by its tiles
  unsigned long long hb, pairs, moves;
  unsigned long long hist[8];
  unsigned int done;           // tiles of the step finished
  unsigned int pad;
};
struct WaveHdr {
  unsigned long long next;     // item counter
  unsigned long long pad0[15]; // alone in its 128-byte line
  unsigned int committed;      // steps of the call committed
  unsigned int abort;          // nonzero: a wait gave up, every block stops
  unsigned int pad1[30];
  WaveMove vring[kWaveRing];
  WaveAcc acc[kWaveRing];
};
// Co-resident blocks of the wavefront kernel for a tile shape (0 if none).
int wave_blocks(int rng_words, bool cmp64, int shape);
// Clears the scratch (scratch_bytes) and launches the call's steps.
cudaError_t launch_wave(const LatticeArgs& A, WaveHdr* H, size_t scratch_bytes, int rng_words,
                        bool cmp64, int shape, long long step0, long long n_steps,
                        const CUtensorMap* tm, cudaStream_t s);

// Host helpers shared by both paths.
void fill_volume_args(const cvf_params* p, long long N, const std::vector<int64_t>& d2,
                      const std::vector<int64_t>& mult, VolumeArgs* va);
bool fill_table24(const cvf_params* p, unsigned long long table24[48]);

}  // namespace cvf
