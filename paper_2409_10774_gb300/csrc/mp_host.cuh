// Host-side internals shared by the C-ABI translation units: the context,
// device buffers, error reporting, problem validation and the per-phase /
// per-axis tables the kernels read.  Nothing here is exported from the
// library.
#pragma once

#include <array>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/micropolar.h"
#include "mp_common.cuh"
#include "mp_plan.cuh"

#define MP_HIDDEN __attribute__((visibility("hidden")))

struct mp_ctx {
  int device = 0;
  int nsm = 1;
  mp_alloc alloc{};
  bool has_alloc = false;
  std::string last_error;
  // launch schedules chosen by the autotuner, per (N1, N2, N3, precision):
  // {pass-A rows per item, fused spectral pass}
  bool autotune = true;
  std::mutex tune_mu;
  std::map<std::array<int, 4>, std::array<int, 2>> tuned;
};

namespace mp {

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Records `fmt` as the last error of `ctx` (and of the calling thread) and returns `st`.
MP_HIDDEN mp_status set_error(mp_ctx* ctx, mp_status st, const char* fmt, ...);
MP_HIDDEN const char* last_error_global();
// Device memory through the context's allocator callbacks, else cudaMalloc.
MP_HIDDEN mp_status dalloc(mp_ctx* ctx, DevBuf& b, size_t bytes);
MP_HIDDEN void dfree(mp_ctx* ctx, DevBuf& b);
// eq. energetic_bounds and the yield parameters of one phase.
MP_HIDDEN mp_status check_phase(const mp_phase& ph, int idx, std::string& msg);
// Full problem validation; fills the phase counts and the reference medium.
MP_HIDDEN mp_status validate_problem(const mp_problem* p, std::vector<long long>* counts_out, double ref[6],
                                     std::string& msg);

// Selects a device for the duration of an entry point and gives the caller's
// current device back when the scope ends.
struct DeviceScope {
  int prev = -1;
  bool changed = false;
  cudaError_t err = cudaSuccess;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) {
      err = cudaSetDevice(dev);
      changed = (err == cudaSuccess) && prev >= 0;
    }
  }
  ~DeviceScope() {
    if (changed) cudaSetDevice(prev);
  }
  DeviceScope(const DeviceScope&) = delete;
  DeviceScope& operator=(const DeviceScope&) = delete;
};

}  // namespace mp

// Opens a DeviceScope on the context's device (returns MP_E_CUDA on failure).
#define MP_DEVICE_SCOPE(ctx)                                                                      \
  ::mp::DeviceScope _mp_dev_scope((ctx)->device);                                                 \
  if (_mp_dev_scope.err != cudaSuccess)                                                           \
  return ::mp::set_error((ctx), MP_E_CUDA, "cudaSetDevice(%d) failed: %s", (ctx)->device,         \
                         cudaGetErrorString(_mp_dev_scope.err))

#define MP_CK(ctx, call)                                                                          \
  do {                                                                                            \
    cudaError_t _e = (call);                                                                      \
    if (_e != cudaSuccess)                                                                        \
      return ::mp::set_error((ctx), _e == cudaErrorMemoryAllocation ? MP_E_OOM : MP_E_CUDA,        \
                             "%s failed: %s (%s:%d)", #call, cudaGetErrorString(_e), __FILE__, __LINE__); \
  } while (0)

// Returns the mp_status of `call` when it is not MP_OK (its error already set).
#define MP_CK_ST(call)                \
  do {                                \
    const mp_status _s = (call);      \
    if (_s != MP_OK) return _s;       \
  } while (0)

namespace mp {

// Per-phase constants of Algorithm 1, prepared in FP64.  ret32 (FP32 fields
// only): the closed-form level return forms its radius, square root, plastic
// multiplier increment and scale factor in FP32 instead of FP64.
template <class R>
PhaseDev<R> phase_dev(const mp_phase& ph, bool ret32 = false) {
  PhaseDev<R> d{};
  d.ret32 = (ret32 && sizeof(R) == 4) ? 1 : 0;
  d.lam = (R)ph.lambda;
  d.mu = (R)ph.mu;
  d.kap = (R)ph.kappa;
  d.alpha = (R)ph.alpha;
  d.beta = (R)ph.beta;
  d.gamma = (R)ph.gamma;
  d.a1 = (R)ph.a1;
  d.a2 = (R)(ph.a1 * ph.mu / ph.kappa);  // Alg. 1: a2 = a1 mu / kappa
  d.b1 = (R)ph.b1;
  d.skew_m = ph.gamma > ph.beta ? 1 : 0;
  d.b2 = d.skew_m ? (R)(ph.b1 * (ph.gamma + ph.beta) / (ph.gamma - ph.beta)) : (R)0;
  d.elastic = ph.elastic ? 1 : 0;
  d.tY = ph.elastic ? INFINITY : ph.tY;
  d.tH = ph.tH;
  d.mY = ph.elastic ? INFINITY : ph.mY;
  d.mH = ph.mH;
  d.tYf = (float)d.tY;
  d.tHf = (float)d.tH;
  d.mYf = (float)d.mY;
  d.mHf = (float)d.mH;
  d.ct = 2.0 * ph.a1 * ph.mu;
  d.cm = ph.b1 * (ph.gamma + ph.beta);
  d.inv_t = 1.0 / (ph.tH + d.ct);
  d.inv_m = 1.0 / (ph.mH + d.cm);
  d.ct_inv = d.ct / (ph.tH + d.ct);
  d.tH_inv = ph.tH / (ph.tH + d.ct);
  d.cm_inv = d.cm / (ph.mH + d.cm);
  d.mH_inv = ph.mH / (ph.mH + d.cm);
  d.inv_tf = (float)d.inv_t;
  d.inv_mf = (float)d.inv_m;
  d.ct_invf = (float)d.ct_inv;
  d.tH_invf = (float)d.tH_inv;
  d.cm_invf = (float)d.cm_inv;
  d.mH_invf = (float)d.mH_inv;
  return d;
}

// The manufactured source of a problem (Appendix D.1) as the kernels read it:
// for each increment s = 1..n_steps, [nvox][18] values t^m - <t^m>,
// m^m - <m^m> in the field type.  The subtracted constants only change the
// zero-frequency term of the polarization, which the Green operator
// discards, so the iterates are those of eq. manufactured_polarization_stress.
template <class R>
void centred_source(const double* tau_m, const double* mu_m, int n_steps, long long nvox, std::vector<R>& out) {
  out.assign((size_t)n_steps * (size_t)nvox * 18, R(0));
  for (int s = 1; s <= n_steps; ++s) {
    const double* ts = tau_m + (size_t)s * nvox * 9;
    const double* ms = mu_m + (size_t)s * nvox * 9;
    double mt[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, mm[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (long long v = 0; v < nvox; ++v)
      for (int q = 0; q < 9; ++q) {
        mt[q] += ts[v * 9 + q];
        mm[q] += ms[v * 9 + q];
      }
    for (int q = 0; q < 9; ++q) {
      mt[q] /= (double)nvox;
      mm[q] /= (double)nvox;
    }
    R* o = out.data() + (size_t)(s - 1) * (size_t)nvox * 18;
    for (long long v = 0; v < nvox; ++v)
      for (int q = 0; q < 9; ++q) {
        o[v * 18 + q] = (R)(ts[v * 9 + q] - mt[q]);
        o[v * 18 + 9 + q] = (R)(ms[v * 9 + q] - mm[q]);
      }
  }
}

template <class R>
RefDev<R> ref_dev(const double ref[6]) {
  RefDev<R> r;
  r.lam = (R)ref[0];
  r.mu = (R)ref[1];
  r.kap = (R)ref[2];
  r.alpha = (R)ref[3];
  r.beta = (R)ref[4];
  r.gamma = (R)ref[5];
  return r;
}

}  // namespace mp
