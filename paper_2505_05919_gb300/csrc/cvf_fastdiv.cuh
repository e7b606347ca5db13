// cvf_fastdiv.cuh -- unsigned division by a value fixed at launch time.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace cvf {

// Unsigned division by an invariant d (1 <= d < 2^31) for any 32-bit n,
// after Granlund and Montgomery, "Division by invariant integers using
// multiplication" (PLDI 1994, Fig. 4.1): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n),
// n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
struct FastDiv {
  uint32_t m, sh1, sh2;
};

inline FastDiv make_fastdiv(uint32_t d) {
  uint32_t l = 0;
  while ((1ull << l) < (unsigned long long)d) ++l;
  FastDiv f;
  f.m = (uint32_t)(((((1ull << l) - d) << 32) / d) + 1);
  f.sh1 = l < 1 ? l : 1;
  f.sh2 = l > 1 ? l - 1 : 0;
  return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  const uint32_t t = __umulhi(f.m, n);
  return (t + ((n - t) >> f.sh1)) >> f.sh2;
}

}  // namespace cvf
