// cvf_batch_nt512.cu -- the batched sweep with 512-thread blocks (half the
// cells per thread of the 256-thread kernels for the same tile), compiled in
// a translation unit of its own so the kernel sets build in parallel.
#include "cvf_batch_kernel.cuh"

namespace cvf {

BatchKernelFn batch_kernel_nt512(int rng_words, bool cmp64, int shape) {
  return batch_kernel_for<512>(rng_words, cmp64, shape);
}

}  // namespace cvf
