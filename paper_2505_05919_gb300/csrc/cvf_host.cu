// cvf_host.cu -- host-side helpers and parameter entry points of the C ABI.
#include <cmath>
#include <cstdio>
#include <cstring>

#include "cvf_device.cuh"
#include "cvf_host.h"

namespace cvf {

static thread_local std::string g_last_error;

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

void clear_error() { g_last_error.clear(); }

int status_error(int status) {
  if (status == 0) return CVF_OK;
  if (status & (int)kStatusBadCell)
    return set_error(CVF_EINVAL, "the lattice holds a word that is not a valid cell for q "
                     "(a nibble >= q or a guard bit set); the result is meaningless");
  if (status >= 0x100)
    return set_error(CVF_EBOUNDS, "a device index check of a debug build failed (site %d)",
                     status - 0x100);
  return set_error(CVF_ETIMEOUT, "a bounded wait in the sweep kernel gave up (status %d)",
                   status);
}

int check_params(const cvf_params* p) {
  if (!p) return set_error(CVF_EINVAL, "params is NULL");
  if (p->L < 2 || (p->L & 1) || p->L > 65534)
    return set_error(CVF_EINVAL, "L=%d: need an even side 2 <= L <= 65534", p->L);
  if (p->q < 2 || p->q > 8)
    return set_error(CVF_EINVAL, "q=%d: need 2 <= q <= 8 (3 bits per arm)", p->q);
  if (!(p->kT > 0.0) || !std::isfinite(p->kT))
    return set_error(CVF_EINVAL, "kT=%g must be positive and finite", p->kT);
  if (!std::isfinite(p->P) || !std::isfinite(p->J) || !std::isfinite(p->J_sigma) ||
      !std::isfinite(p->v_HB) || !std::isfinite(p->epsilon))
    return set_error(CVF_EINVAL, "energies, P and v_HB must be finite");
  if (!(p->cutoff > 0.0) || p->cutoff > 16.0)
    return set_error(CVF_EINVAL, "cutoff=%g must be in (0, 16] r0", p->cutoff);
  if (!(p->v_iso_init >= 1.0) || !std::isfinite(p->v_iso_init))
    return set_error(CVF_EINVAL, "v_iso_init=%g must be >= 1 (hard core)", p->v_iso_init);
  if (!(p->dv_max_frac >= 0.0) || !std::isfinite(p->dv_max_frac))
    return set_error(CVF_EINVAL, "dv_max_frac=%g must be >= 0", p->dv_max_frac);
  if (p->init != CVF_INIT_RANDOM && p->init != CVF_INIT_ORDERED)
    return set_error(CVF_EINVAL, "init=%d unknown", p->init);
  if (p->schedule != CVF_SCHED_CHECKERBOARD && p->schedule != CVF_SCHED_LAYERED)
    return set_error(CVF_EINVAL, "schedule=%d unknown", p->schedule);
  if (p->volume_moves != 0 && p->volume_moves != 1)
    return set_error(CVF_EINVAL, "volume_moves=%d must be 0 or 1", p->volume_moves);
  if (p->rng_words != 1 && p->rng_words != 2)
    return set_error(CVF_EINVAL, "rng_words=%d must be 1 or 2", p->rng_words);
  if (p->eta_moves != 0)
    return set_error(CVF_EINVAL, "eta_moves=%d: the square lattice has eta = 1 on every edge "
                     "(four neighbours per cell); eta moves exist on the cubic lattice only",
                     p->eta_moves);
  return CVF_OK;
}

void threshold_table(const cvf_params* p, uint64_t out[42]) {
  const double J_eff = p->J - p->P * p->v_HB;
  for (int g = 0; g < 2; ++g)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 7; ++j) {
        const int dhb = i - 1, dc = j - 3;
        const double dH = -((double)g * J_eff) * (double)dhb - p->J_sigma * (double)dc;
        uint64_t t;
        if (dH <= 0.0)
          t = (uint64_t)1 << 32;
        else
          t = (uint64_t)(std::exp(-dH / p->kT) * 4294967296.0);
        out[(g * 3 + i) * 7 + j] = t;
      }
}

void lattice_shells(double cutoff, std::vector<int64_t>* d2, std::vector<int64_t>* mult) {
  d2->clear();
  mult->clear();
  const int R = (int)std::ceil(cutoff);
  // count lattice vectors per squared length, then keep those inside the cutoff
  std::vector<int64_t> count((size_t)2 * R * R + 1, 0);
  for (int i = -R; i <= R; ++i)
    for (int j = -R; j <= R; ++j) {
      const int64_t s = (int64_t)i * i + (int64_t)j * j;
      if (s > 0) count[(size_t)s] += 1;
    }
  for (size_t s = 1; s < count.size(); ++s)
    if (count[s] > 0 && (double)s < cutoff * cutoff) {
      d2->push_back((int64_t)s);
      mult->push_back(count[s]);
    }
}

int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}

}  // namespace cvf

extern "C" {

const char* cvf_last_error(void) { return cvf::g_last_error.c_str(); }

int cvf_params_default(cvf_params* out) { return cvf_params_physical(300.0, 0.1, out); }

int cvf_params_physical(double T_kelvin, double P_MPa, cvf_params* out) {
  if (!out) return cvf::set_error(CVF_EINVAL, "out is NULL");
  if (!(T_kelvin > 0.0) || !std::isfinite(T_kelvin) || !std::isfinite(P_MPa))
    return cvf::set_error(CVF_EINVAL, "T=%g K, P=%g MPa: need T > 0 and finite P", T_kelvin,
                          P_MPa);
  // Table 1: eps = 5.5 kJ/mol, r0 = 2.9 Angstrom, v0 = r0^3.
  const double R = 8.31446261815324e-3;  // kJ / (mol K)
  const double eps = 5.5;                // kJ / mol
  const double r0 = 2.9e-10;             // m
  const double NA = 6.02214076e23;       // 1 / mol
  std::memset(out, 0, sizeof(*out));
  out->L = 64;
  out->q = 6;
  out->epsilon = 1.0;
  out->cutoff = 6.0;
  out->J = 2.0;        // J/(4 eps) = 0.5
  out->J_sigma = 0.32; // J_sigma/(4 eps) = 0.08
  out->v_HB = 0.6;
  out->kT = T_kelvin * R / eps;
  out->P = (P_MPa * 1.0e6) * (r0 * r0 * r0) * NA / (eps * 1.0e3);
  out->v_iso_init = std::cbrt(2.0);
  out->dv_max_frac = 0.01;
  out->seed = 1;
  out->init = CVF_INIT_RANDOM;
  out->schedule = CVF_SCHED_CHECKERBOARD;
  out->volume_moves = 1;
  out->rng_words = 1;
  return CVF_OK;
}

int cvf_threshold_table(const cvf_params* p, uint64_t out[42]) {
  if (!out) return cvf::set_error(CVF_EINVAL, "out is NULL");
  const int rc = cvf::check_params(p);
  if (rc) return rc;
  cvf::threshold_table(p, out);
  return CVF_OK;
}

int cvf_debug_checks(void) {
#ifdef CVF_DEBUG
  return 1;
#else
  return 0;
#endif
}

}  // extern "C"
