// cvf_lattice.cuh -- launch arguments of the single-lattice kernels.
#pragma once
#include <cstdint>

#include "cvf_device.cuh"

namespace cvf {

constexpr int kThreads = 256;

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
};

}  // namespace cvf
