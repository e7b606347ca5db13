// cvf_host.h -- host-side helpers of the CVF library: thread-local error
// text, CUDA status checks, parameter validation, threshold and shell tables.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include "cvf.h"

namespace cvf {

int set_error(int code, const char* fmt, ...);
void clear_error();

#define CVF_CUDA_CHECK(expr)                                                   \
  do {                                                                         \
    cudaError_t e_ = (expr);                                                   \
    if (e_ != cudaSuccess)                                                     \
      return ::cvf::set_error(CVF_ECUDA, "%s failed: %s (%s:%d)", #expr,       \
                              cudaGetErrorString(e_), __FILE__, __LINE__);     \
  } while (0)

// Validation shared by every creation path; returns CVF_OK or CVF_EINVAL
// with the reason recorded.
int check_params(const cvf_params* p);

// The 42 thresholds [g][dN_HB+1][dN_sigma+3] (Sec. II.C with Eq. H).
void threshold_table(const cvf_params* p, uint64_t out[42]);

// Shells of the square lattice inside the cutoff at the hard-core density:
// squared lengths (ascending) and the number of lattice vectors in each.
void lattice_shells(double cutoff, std::vector<int64_t>* d2,
                    std::vector<int64_t>* mult);

int sm_count();

// The status word of a lattice's observables as a call result: 0 CVF_OK,
// 1 CVF_ETIMEOUT (a bounded device wait gave up), 0x100 + site CVF_EBOUNDS
// (a debug build's index check failed at `site`), bit 0x200 CVF_EINVAL (the
// lattice held a word that is not a valid cell).
int status_error(int status);

// An NVTX range over one host entry point, named after it, so that a
// profiler that records NVTX (ncu --nvtx, a timeline tracer) can attribute the
// launches to the API call that made them; without one attached the push and
// pop return at once.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace cvf
