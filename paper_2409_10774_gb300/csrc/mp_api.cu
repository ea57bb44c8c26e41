// C ABI of the micropolar FFT solver: validation, device state, and the
// host-side load-step / fixed-point loop of Algorithm 2 around the kernels.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/micropolar.h"
#include "mp_host.cuh"
#include "mp_kernels.cuh"

using namespace mp;

namespace mp {

namespace {
thread_local std::string g_last_error;
}  // namespace

mp_status set_error(mp_ctx* ctx, mp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->last_error = buf;
  g_last_error = buf;
  return st;
}

const char* last_error_global() { return g_last_error.c_str(); }

}  // namespace mp

namespace mp {

// ------------------------------------------------------------------ device memory
mp_status dalloc(mp_ctx* ctx, DevBuf& b, size_t bytes) {
  b.bytes = bytes;
  b.ptr = nullptr;
  if (bytes == 0) return MP_OK;
  if (ctx->has_alloc && ctx->alloc.alloc) {
    b.ptr = ctx->alloc.alloc(bytes, ctx->alloc.user);
    if (!b.ptr) return set_error(ctx, MP_E_OOM, "device allocation of %zu bytes failed", bytes);
    return MP_OK;
  }
  cudaError_t e = cudaMalloc(&b.ptr, bytes);
  if (e != cudaSuccess) {
    b.ptr = nullptr;
    return set_error(ctx, MP_E_OOM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
  }
  return MP_OK;
}

void dfree(mp_ctx* ctx, DevBuf& b) {
  if (!b.ptr) return;
  if (ctx->has_alloc && ctx->alloc.free) ctx->alloc.free(b.ptr, b.bytes, ctx->alloc.user);
  else if (!ctx->has_alloc) cudaFree(b.ptr);
  b.ptr = nullptr;
  b.bytes = 0;
}

// ------------------------------------------------------------------ validation
static bool size_ok(int n) {
  if (n == 1) return true;
  if (n < 2 || n > 512 || (n % 2) != 0) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

static bool finite(double v) { return std::isfinite(v); }

mp_status check_phase(const mp_phase& ph, int idx, std::string& msg) {
  const double v[12] = {ph.lambda, ph.mu, ph.kappa, ph.alpha, ph.beta, ph.gamma,
                        ph.tY, ph.tH, ph.mY, ph.mH, ph.a1, ph.b1};
  for (double x : v)
    if (!finite(x)) {
      msg = "phase " + std::to_string(idx) + ": non-finite parameter";
      return MP_E_INVALID_ARG;
    }
  // eq. energetic_bounds, with gamma - beta >= 0 (equality: the skew couple stress vanishes)
  if (!(3 * ph.lambda + 2 * ph.mu > 0) || !(ph.mu > 0) || !(ph.kappa > 0) ||
      !(3 * ph.alpha + ph.beta + ph.gamma > 0) || !(ph.gamma + ph.beta > 0) || !(ph.gamma - ph.beta >= 0)) {
    msg = "phase " + std::to_string(idx) + ": moduli violate the energetic bounds";
    return MP_E_INADMISSIBLE;
  }
  if (!ph.elastic) {
    if (!(ph.tY > 0) || !(ph.mY > 0) || !(ph.tH >= 0) || !(ph.mH >= 0) || !(ph.a1 > 0) || !(ph.b1 > 0)) {
      msg = "phase " + std::to_string(idx) + ": need tY, mY, a1, b1 > 0 and tH, mH >= 0";
      return MP_E_INVALID_ARG;
    }
  } else if (!(ph.a1 > 0) || !(ph.b1 > 0)) {
    msg = "phase " + std::to_string(idx) + ": need a1, b1 > 0";
    return MP_E_INVALID_ARG;
  }
  return MP_OK;
}

// Reference medium (6 moduli) over the phases present in the map.
static mp_status reference_moduli(const mp_problem* p, const std::vector<long long>& counts, long long nvox,
                           double ref[6], std::string& msg) {
  if (p->ref_kind == MP_REF_EXPLICIT) {
    if (!p->ref_moduli) {
      msg = "ref_moduli required for MP_REF_EXPLICIT";
      return MP_E_INVALID_ARG;
    }
    for (int i = 0; i < 6; ++i) ref[i] = p->ref_moduli[i];
  } else {
    for (int i = 0; i < 6; ++i) ref[i] = (p->ref_kind == MP_REF_MEAN) ? 0.0 : NAN;
    double lo[6], hi[6];
    for (int i = 0; i < 6; ++i) {
      lo[i] = INFINITY;
      hi[i] = -INFINITY;
    }
    for (int k = 0; k < p->n_phases; ++k) {
      if (counts[k] == 0) continue;
      const mp_phase& ph = p->phases[k];
      const double m[6] = {ph.lambda, ph.mu, ph.kappa, ph.alpha, ph.beta, ph.gamma};
      for (int i = 0; i < 6; ++i) {
        if (p->ref_kind == MP_REF_MEAN) ref[i] += m[i] * (double)counts[k];
        lo[i] = std::fmin(lo[i], m[i]);
        hi[i] = std::fmax(hi[i], m[i]);
      }
    }
    for (int i = 0; i < 6; ++i)
      ref[i] = (p->ref_kind == MP_REF_MEAN) ? ref[i] / (double)nvox : 0.5 * (lo[i] + hi[i]);
  }
  for (int i = 0; i < 6; ++i)
    if (!finite(ref[i])) {
      msg = "reference moduli not finite";
      return MP_E_INVALID_ARG;
    }
  // the Green operator needs lam0 + 2 mu0, mu0, kappa0 > 0 and gamma0, alpha0 + beta0 + gamma0 >= 0
  if (!(ref[0] + 2 * ref[1] > 0) || !(ref[1] > 0) || !(ref[2] > 0) || !(ref[5] >= 0) ||
      !(ref[3] + ref[4] + ref[5] >= 0)) {
    msg = "reference medium not admissible for the Green operator";
    return MP_E_INADMISSIBLE;
  }
  return MP_OK;
}

mp_status validate_problem(const mp_problem* p, std::vector<long long>* counts_out, double ref[6],
                           std::string& msg) {
  if (!p) {
    msg = "problem is NULL";
    return MP_E_INVALID_ARG;
  }
  for (int j = 0; j < 3; ++j)
    if (p->n[j] < 1) {
      msg = "grid sizes must be >= 1";
      return MP_E_INVALID_ARG;
    }
  for (int j = 0; j < 3; ++j)
    if (!size_ok(p->n[j])) {
      msg = "grid size " + std::to_string(p->n[j]) + " unsupported (1 or even 2^a 3^b <= 512)";
      return MP_E_UNSUPPORTED_SIZE;
    }
  if (!(p->h > 0) || !finite(p->h)) {
    msg = "voxel size h must be positive";
    return MP_E_INVALID_ARG;
  }
  if (!p->phase || !p->phases || p->n_phases < 1 || p->n_phases > 65536) {
    msg = "phase map / phase table missing";
    return MP_E_INVALID_ARG;
  }
  for (int k = 0; k < p->n_phases; ++k) {
    mp_status st = check_phase(p->phases[k], k, msg);
    if (st != MP_OK) return st;
  }
  if (p->n_steps < 1 || !p->time || !p->E || !p->G) {
    msg = "load path missing";
    return MP_E_INVALID_ARG;
  }
  for (int s = 0; s <= p->n_steps; ++s) {
    if (!finite(p->time[s])) {
      msg = "time not finite";
      return MP_E_INVALID_ARG;
    }
    if (s > 0 && !(p->time[s] > p->time[s - 1])) {
      msg = "time must be strictly increasing";
      return MP_E_INVALID_ARG;
    }
    for (int q = 0; q < 9; ++q)
      if (!finite(p->E[9 * s + q]) || !finite(p->G[9 * s + q])) {
        msg = "load path not finite";
        return MP_E_INVALID_ARG;
      }
  }
  if (!(p->tol > 0) || !finite(p->tol)) {
    msg = "tol must be positive";
    return MP_E_INVALID_ARG;
  }
  if (p->err_kind != MP_ERR_LOCAL && p->err_kind != MP_ERR_AVERAGE) {
    msg = "err_kind must be 0 or 1";
    return MP_E_INVALID_ARG;
  }
  if (p->ref_kind < 0 || p->ref_kind > 2) {
    msg = "ref_kind must be 0, 1 or 2";
    return MP_E_INVALID_ARG;
  }
  if (p->precision < 0 || p->precision > 2) {
    msg = "precision must be 0, 1 or 2";
    return MP_E_INVALID_ARG;
  }
  if (!(p->precision == 0 ? sizes_fit<double>(p->n[0], p->n[1], p->n[2])
                          : sizes_fit<float>(p->n[0], p->n[1], p->n[2]))) {
    msg = "grid too large for the kernels' shared-memory tiles at this precision";
    return MP_E_UNSUPPORTED_SIZE;
  }
  if ((p->tau_m == nullptr) != (p->mu_m == nullptr)) {
    msg = "tau_m and mu_m must be given together";
    return MP_E_INVALID_ARG;
  }
  if (p->tau_m) {
    const size_t nsrc = (size_t)(p->n_steps + 1) * (size_t)p->n[0] * p->n[1] * p->n[2] * 9;
    for (size_t i = 0; i < nsrc; ++i)
      if (!finite(p->tau_m[i]) || !finite(p->mu_m[i])) {
        msg = "manufactured source not finite";
        return MP_E_INVALID_ARG;
      }
  }
  if (p->lockstep_iters)
    for (int s = 0; s < p->n_steps; ++s)
      if (p->lockstep_iters[s] < 1) {
        msg = "lockstep iteration counts must be >= 1";
        return MP_E_INVALID_ARG;
      }
  const long long nvox = (long long)p->n[0] * p->n[1] * p->n[2];
  std::vector<long long> counts(p->n_phases, 0);
  for (long long v = 0; v < nvox; ++v) {
    const int id = p->phase[v];
    if (id >= p->n_phases) {
      msg = "phase id " + std::to_string(id) + " out of range";
      return MP_E_INVALID_ARG;
    }
    counts[id]++;
  }
  mp_status st = reference_moduli(p, counts, nvox, ref, msg);
  if (st != MP_OK) return st;
  if (counts_out) *counts_out = std::move(counts);
  return MP_OK;
}

// ------------------------------------------------------------------ plans and tables
template <class R>
mp_status make_axis(mp_ctx* ctx, int n, bool packed, AxisPlan<R>& p, DevBuf& tw, cudaStream_t st,
                    std::vector<cpx<R>>& host_tw) {
  axis_tables<R>(n, packed, p, host_tw);
  mp_status s = dalloc(ctx, tw, sizeof(cpx<R>) * n);
  if (s != MP_OK) return s;
  MP_CK(ctx, cudaMemcpyAsync(tw.ptr, host_tw.data(), sizeof(cpx<R>) * n, cudaMemcpyHostToDevice, st));
  p.tw = reinterpret_cast<const cpx<R>*>(tw.ptr);
  return MP_OK;
}


}  // namespace mp

// ------------------------------------------------------------------ cell state
struct mp_rve {
  mp_ctx* ctx = nullptr;
  int precision = 1;
  int n[3] = {1, 1, 1};
  long long nvox = 0, nspec = 0;
  double h = 1.0;
  int n_steps = 0;
  std::vector<double> time, E, G;
  double tol = 1e-6;
  int err_kind = 0, max_iter = 10000;
  std::vector<int> lockstep;
  double div_limit = 1e6;
  double ref[6] = {0, 0, 0, 0, 0, 0};
  DevBuf spec, prev, hist, pq, elast, phase, phases, twx, twy, twz, partials, avgpart, errout, steprows,
      status, tmean, ctl, src;
  CellDev<float> cf{};
  CellDev<double> cd{};
  LaunchCfg L;
  int steps_done = 0;
  bool predicted = false;
  long long total_iters = 0;
  int failed_step = 0;
  std::vector<double> err_steps;
  std::vector<int> iters_steps;
  double* err_host = nullptr;  // pinned, 16 doubles
  uint64_t digest = 0;         // of the problem the cell was created from (checkpoint check)
  // per-kernel-class launch counters and (when profiling) CUDA-event timings
  long long launches[MP_KC_COUNT] = {0};
  double kernel_ms[MP_KC_COUNT] = {0};
  bool profiling = false;
  // convergence trace: (step, iteration, err, err_e, err_t, err_gamma, err_m) per iteration
  bool tracing = false;
  std::vector<double> trace;
  cudaEvent_t ev[2 * MP_KC_COUNT] = {};
  // device-decided fixed-point loop (CUDA graph with a conditional WHILE node)
  cudaStream_t capture = nullptr;  // private stream the loop graph is captured on
  bool device_loop = true;         // false once a graph call failed (then the host decides)
  bool use_fused = true;           // the fused spectral pass, where the cell has one (autotuner's choice)
  bool tuned = false;              // launch schedule chosen by timing candidates
  // loop bounds of the next device-decided loop: iteration budget and the
  // stagnation window (0: no watch)
  int loop_budget = 0, loop_stag = 0, loop_adapt = 0;
  // FP32-mixed increments whose iteration stalls above the tolerance
  // (precision 1 without a prescribed schedule) continue in the increment
  // form and, if that stalls too, finish in FP64: FP64 copies of the
  // precision-dependent state (cell cd), allocated at the first such increment.
  std::vector<mp_phase> phases_host;
  DevBuf spec64, prev64, hist64, elast64, phases64, twx64, twy64, twz64, partials64, avgpart64;
  LaunchCfg L64;
  bool twin = false;
  std::vector<int> iters64_steps;  // iterations of each increment run in FP64
  long long delta_switches = 0, escalations = 0;
  bool skip_delta = false;  // the increment form stalled once: later stalls go to FP64 directly
};

namespace {

template <class R>
CellDev<R>& cell_of(mp_rve* r);
template <>
CellDev<float>& cell_of<float>(mp_rve* r) { return r->cf; }
template <>
CellDev<double>& cell_of<double>(mp_rve* r) { return r->cd; }

// Launch configuration and reduction buffers of the cell of type R: the
// cell's own, or those of the FP64 copy of an FP32-mixed cell.
template <class R>
LaunchCfg& cfg_of(mp_rve* r) { return (sizeof(R) == 8 && r->precision != 0) ? r->L64 : r->L; }
template <class R>
double* partials_of(mp_rve* r) {
  return reinterpret_cast<double*>((sizeof(R) == 8 && r->precision != 0) ? r->partials64.ptr : r->partials.ptr);
}
template <class R>
double* avgpart_of(mp_rve* r) {
  return reinterpret_cast<double*>((sizeof(R) == 8 && r->precision != 0) ? r->avgpart64.ptr : r->avgpart.ptr);
}

template <class R>
mp_status rve_setup(mp_rve* r, const mp_problem* p, cudaStream_t st) {
  mp_ctx* ctx = r->ctx;
  CellDev<R>& c = cell_of<R>(r);
  c = CellDev<R>{};
  c.n1 = p->n[0];
  c.n2 = p->n[1];
  c.n3 = p->n[2];
  c.kx = (c.n1 > 1) ? c.n1 / 2 : 1;
  c.nvox = r->nvox;
  c.nspec = (long long)c.kx * c.n2 * c.n3;
  r->nspec = c.nspec;
  c.h = p->h;
  c.inv_nvox = 1.0 / (double)r->nvox;
  for (int j = 0; j < 3; ++j) c.two_pi_over_L[j] = (R)(2.0 * M_PI / ((double)p->n[j] * p->h));
  mp_status s;
  if ((s = dalloc(ctx, r->spec, sizeof(cpx<R>) * 18 * (size_t)c.nspec)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->prev, sizeof(R) * 20 * (size_t)c.nvox)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->hist, sizeof(R) * 20 * (size_t)c.nvox)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->status, sizeof(int) * 4)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->tmean, sizeof(double) * kCellScalars)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->pq, sizeof(double) * 2 * (size_t)c.nvox)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->elast, sizeof(R) * 18 * (size_t)c.nvox)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->phase, sizeof(uint16_t) * (size_t)c.nvox)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->phases, sizeof(PhaseDev<R>) * (size_t)p->n_phases)) != MP_OK) return s;
  c.spec = reinterpret_cast<cpx<R>*>(r->spec.ptr);
  c.prev = reinterpret_cast<R*>(r->prev.ptr);
  c.hist = reinterpret_cast<R*>(r->hist.ptr);
  c.pq = reinterpret_cast<double*>(r->pq.ptr);
  c.elast = reinterpret_cast<R*>(r->elast.ptr);
  c.phase = reinterpret_cast<const uint16_t*>(r->phase.ptr);
  c.phases = reinterpret_cast<const PhaseDev<R>*>(r->phases.ptr);
  c.status = reinterpret_cast<int*>(r->status.ptr);
  c.tmean = reinterpret_cast<double*>(r->tmean.ptr);
  c.err_kind = r->err_kind;
  MP_CK(ctx, cudaMemsetAsync(r->status.ptr, 0, r->status.bytes, st));
  MP_CK(ctx, cudaMemsetAsync(r->tmean.ptr, 0, r->tmean.bytes, st));
  c.ref = ref_dev<R>(r->ref);
  std::vector<PhaseDev<R>> ph(p->n_phases);
  for (int k = 0; k < p->n_phases; ++k) ph[k] = phase_dev<R>(p->phases[k], p->precision == 2);
  std::vector<cpx<R>> t1, t2, t3;
  if ((s = make_axis<R>(ctx, c.n1, true, c.px, r->twx, st, t1)) != MP_OK) return s;
  if ((s = make_axis<R>(ctx, c.n2, false, c.py, r->twy, st, t2)) != MP_OK) return s;
  if ((s = make_axis<R>(ctx, c.n3, false, c.pz, r->twz, st, t3)) != MP_OK) return s;
  MP_CK(ctx, cudaMemcpyAsync(r->phase.ptr, p->phase, sizeof(uint16_t) * (size_t)c.nvox,
                             cudaMemcpyHostToDevice, st));
  MP_CK(ctx, cudaMemcpyAsync(r->phases.ptr, ph.data(), sizeof(PhaseDev<R>) * ph.size(),
                             cudaMemcpyHostToDevice, st));
  r->L = make_launch_cfg<R>(c, ctx->nsm);
  c.rows_a = r->L.rows;
  c.items_a = r->L.items_a;
  // per-block error partials for the largest pass-A grid any schedule can take
  // (pass A keeps at most two blocks on an SM)
  const size_t max_grid = std::max<size_t>((size_t)r->L.grid_a, 2 * (size_t)ctx->nsm);
  if ((s = dalloc(ctx, r->partials, sizeof(double) * kErrPartials * max_grid)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->avgpart, sizeof(double) * kAvgPartials * (size_t)r->L.grid_v)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->errout, sizeof(double) * 16)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->steprows, sizeof(double) * kAvgPartials * (size_t)r->n_steps)) != MP_OK) return s;
  std::vector<R> src_host;
  if (p->tau_m) {
    centred_source<R>(p->tau_m, p->mu_m, p->n_steps, r->nvox, src_host);
    if ((s = dalloc(ctx, r->src, sizeof(R) * src_host.size())) != MP_OK) return s;
    MP_CK(ctx, cudaMemcpyAsync(r->src.ptr, src_host.data(), sizeof(R) * src_host.size(), cudaMemcpyHostToDevice, st));
  }
  if constexpr (sizeof(R) == 4) {
    if (spectral_fused_ok(c)) {
      if ((s = dalloc(ctx, r->ctl, sizeof(int) * spectral_ctl_ints(c.kx))) != MP_OK) return s;
      MP_CK(ctx, cudaMemsetAsync(r->ctl.ptr, 0, r->ctl.bytes, st));
    }
  }
  MP_CK(ctx, cudaMemsetAsync(r->steprows.ptr, 0, r->steprows.bytes, st));
  // host tables are stack-local: finish the uploads before returning
  MP_CK(ctx, cudaStreamSynchronize(st));
  return MP_OK;
}

// The FP64 copy of an FP32-mixed cell: its own spectrum, records, phase
// table, twiddles and reduction buffers; the FP64 state (p, q), the cell
// scalars, the phase map, the status word and the result rows are shared
// with the FP32 cell.
mp_status twin_setup(mp_rve* r, cudaStream_t st) {
  if (r->twin) return MP_OK;
  mp_ctx* ctx = r->ctx;
  const CellDev<float>& f = r->cf;
  CellDev<double>& c = r->cd;
  c = CellDev<double>{};
  c.n1 = f.n1;
  c.n2 = f.n2;
  c.n3 = f.n3;
  c.kx = f.kx;
  c.nvox = f.nvox;
  c.nspec = f.nspec;
  c.h = f.h;
  c.inv_nvox = f.inv_nvox;
  for (int j = 0; j < 3; ++j) c.two_pi_over_L[j] = 2.0 * M_PI / ((double)r->n[j] * r->h);
  mp_status s;
  if ((s = dalloc(ctx, r->spec64, sizeof(cpx<double>) * 18 * (size_t)c.nspec)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->prev64, sizeof(double) * 20 * (size_t)c.nvox)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->hist64, sizeof(double) * 20 * (size_t)c.nvox)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->elast64, sizeof(double) * 18 * (size_t)c.nvox)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->phases64, sizeof(PhaseDev<double>) * r->phases_host.size())) != MP_OK) return s;
  c.spec = reinterpret_cast<cpx<double>*>(r->spec64.ptr);
  c.prev = reinterpret_cast<double*>(r->prev64.ptr);
  c.hist = reinterpret_cast<double*>(r->hist64.ptr);
  c.elast = reinterpret_cast<double*>(r->elast64.ptr);
  c.phases = reinterpret_cast<const PhaseDev<double>*>(r->phases64.ptr);
  c.pq = f.pq;
  c.phase = f.phase;
  c.status = f.status;
  c.tmean = f.tmean;
  c.err_kind = r->err_kind;
  c.ref = ref_dev<double>(r->ref);
  std::vector<PhaseDev<double>> ph(r->phases_host.size());
  for (size_t k = 0; k < ph.size(); ++k) ph[k] = phase_dev<double>(r->phases_host[k], false);
  std::vector<cpx<double>> t1, t2, t3;
  if ((s = make_axis<double>(ctx, c.n1, true, c.px, r->twx64, st, t1)) != MP_OK) return s;
  if ((s = make_axis<double>(ctx, c.n2, false, c.py, r->twy64, st, t2)) != MP_OK) return s;
  if ((s = make_axis<double>(ctx, c.n3, false, c.pz, r->twz64, st, t3)) != MP_OK) return s;
  MP_CK(ctx, cudaMemcpyAsync(r->phases64.ptr, ph.data(), sizeof(PhaseDev<double>) * ph.size(),
                             cudaMemcpyHostToDevice, st));
  r->L64 = make_launch_cfg<double>(c, ctx->nsm);
  c.rows_a = r->L64.rows;
  c.items_a = r->L64.items_a;
  const size_t max_grid = std::max<size_t>((size_t)r->L64.grid_a, 2 * (size_t)ctx->nsm);
  if ((s = dalloc(ctx, r->partials64, sizeof(double) * kErrPartials * max_grid)) != MP_OK) return s;
  if ((s = dalloc(ctx, r->avgpart64, sizeof(double) * kAvgPartials * (size_t)r->L64.grid_v)) != MP_OK) return s;
  MP_CK(ctx, cudaStreamSynchronize(st));  // the host tables are locals
  r->twin = true;
  return MP_OK;
}

template <class R>
void set_load(CellDev<R>& c, const mp_rve* r, int s) {
  for (int q = 0; q < 9; ++q) {
    c.E[q] = (R)r->E[9 * s + q];
    c.G[q] = (R)r->G[9 * s + q];
  }
}

// The kernels of one fixed-point iteration (Algorithm 2's loop body), with
// the loop-deciding error reduction when `handle` is given.
template <class R>
cudaError_t launch_iteration_kernels(mp_rve* r, CellDev<R>& c, cudaStream_t st, const cudaGraphConditionalHandle* handle) {
  const LaunchCfg& L = cfg_of<R>(r);
  double* parts = partials_of<R>(r);
  double* eout = reinterpret_cast<double*>(r->errout.ptr);
  cudaError_t e = cudaSuccess;
  bool fused = false;
  if constexpr (sizeof(R) == 4) fused = r->use_fused && r->ctl.ptr != nullptr;
  if (fused) {
    if constexpr (sizeof(R) == 4) e = launch_spectral(c, reinterpret_cast<int*>(r->ctl.ptr), r->ctx->nsm, st);
  } else {
    e = launch_fft_y<R>(L, c, -1, st);
    if (e == cudaSuccess) e = launch_green_z<R>(L, c, st);
    if (e == cudaSuccess) e = launch_fft_y<R>(L, c, +1, st);
  }
  if (e == cudaSuccess) e = launch_pass_a_iter<R>(L, c, parts, st);
  if (e != cudaSuccess) return e;
  if (handle)
    return launch_reduce_err_loop<R>(L, c, parts, r->err_kind, eout, r->tol, r->loop_budget, r->div_limit,
                                     r->loop_stag, r->loop_adapt, *handle, st);
  return launch_reduce_err<R>(L, c, parts, r->err_kind, eout, st);
}

// Algorithm 2's while loop of one increment decided on the device: a graph
// whose conditional WHILE node repeats the iteration kernels while the error
// reduction finds err > tol (and no failure, fewer than r->loop_budget
// iterations, no stall under a window r->loop_stag > 0), launched once; the
// host reads the outcome (out[0..9]) after it ends.
// Returns cudaErrorNotSupported (nothing launched) when a graph call fails.
template <class R>
cudaError_t device_loop(mp_rve* r, CellDev<R>& c, cudaStream_t st, int& it, double* out) {
  if (!r->capture && cudaStreamCreateWithFlags(&r->capture, cudaStreamNonBlocking) != cudaSuccess) {
    r->capture = nullptr;
    return cudaErrorNotSupported;
  }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return cudaErrorNotSupported;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);  // err(1) = 2 tol: enter once
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  if (e == cudaSuccess) {
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(r->capture, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      const cudaError_t el = launch_iteration_kernels<R>(r, c, r->capture, &h);
      e = cudaStreamEndCapture(r->capture, &body);
      if (e == cudaSuccess) e = el;
    }
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (ge) cudaGraphExecDestroy(ge);
    cudaGraphDestroy(g);
    return cudaErrorNotSupported;
  }
  double* eout = reinterpret_cast<double*>(r->errout.ptr);
  // loop count and stagnation watch from zero; the longest gap between lows
  // (out[10]) carried in from the increment's earlier stages
  e = cudaMemsetAsync(eout + 6, 0, sizeof(double) * 4, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(eout + 10, out + 10, sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaGraphLaunch(ge, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, eout, sizeof(double) * 11, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaGraphExecDestroy(ge);
  cudaGraphDestroy(g);
  if (e == cudaSuccess) it = (int)out[6];
  return e;
}

// Launch-schedule autotuner.  Candidates: pass A with the default rows per
// item, half and a quarter of them (a smaller tile per block, more blocks),
// and, for cells with a fused spectral pass, that pass or the three separate
// column passes.  Each is timed (CUDA events) over three fixed-point
// iterations of the cell's first load increment after one untimed; the
// fastest is kept for the cell and cached in the context for its shape and
// precision.  The cell is then reset to its zero state (the solve starts
// from k_init as always).  Schedules differ only in how the work is split,
// so results agree to rounding (the error partials are summed in another
// order).
template <class R>
mp_status rve_autotune(mp_rve* r, cudaStream_t st) {
  mp_ctx* ctx = r->ctx;
  CellDev<R>& c = cell_of<R>(r);
  const int rows0 = r->L.rows;
  std::vector<int> rows_c{rows0};
  for (int d : {2, 4})
    if (rows0 / d >= 1 && std::find(rows_c.begin(), rows_c.end(), rows0 / d) == rows_c.end()) rows_c.push_back(rows0 / d);
  std::vector<int> fused_c{0};
  if (r->ctl.ptr) fused_c = {1, 0};
  const std::array<int, 4> key{r->n[0], r->n[1], r->n[2], r->precision};
  auto apply = [&](int rows, int fused) {
    r->L = make_launch_cfg<R>(c, ctx->nsm, rows);
    c.rows_a = r->L.rows;
    c.items_a = r->L.items_a;
    r->use_fused = fused != 0;
  };
  {
    std::lock_guard<std::mutex> lock(ctx->tune_mu);
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) {
      apply(it->second[0], it->second[1]);
      r->tuned = true;
      return MP_OK;
    }
  }
  if (rows_c.size() * fused_c.size() < 2) return MP_OK;
  cudaEvent_t e0, e1;
  MP_CK(ctx, cudaEventCreate(&e0));
  MP_CK(ctx, cudaEventCreate(&e1));
  set_load(c, r, 1);
  c.src = r->src.ptr ? reinterpret_cast<const R*>(r->src.ptr) : nullptr;
  float best = INFINITY;
  int best_rows = rows0, best_fused = fused_c[0];
  cudaError_t err = launch_start<R>(r->L, c, 1, st);
  for (int fused : fused_c)
    for (int rows : rows_c) {
      if (err != cudaSuccess) break;
      apply(rows, fused);
      err = launch_iteration_kernels<R>(r, c, st, nullptr);
      if (err == cudaSuccess) err = cudaEventRecord(e0, st);
      for (int k = 0; k < 3 && err == cudaSuccess; ++k) err = launch_iteration_kernels<R>(r, c, st, nullptr);
      if (err == cudaSuccess) err = cudaEventRecord(e1, st);
      if (err == cudaSuccess) err = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
      if (err == cudaSuccess && ms < best) {
        best = ms;
        best_rows = rows;
        best_fused = fused;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  MP_CK(ctx, err);
  apply(best_rows, best_fused);
  // back to the zero state
  MP_CK(ctx, cudaMemsetAsync(r->tmean.ptr, 0, r->tmean.bytes, st));
  MP_CK(ctx, cudaMemsetAsync(r->status.ptr, 0, r->status.bytes, st));
  MP_CK(ctx, cudaStreamSynchronize(st));
  r->tuned = true;
  std::lock_guard<std::mutex> lock(ctx->tune_mu);
  ctx->tuned[key] = {best_rows, best_fused};
  return MP_OK;
}

// Outcome of one stage of an increment's fixed-point loop.
struct LoopOut {
  int it = 0;                // iterations run by the stage
  double err = 0.0;          // error of its last iteration
  bool stalled = false;      // ended by the stagnation watch
  mp_status status = MP_OK;  // MP_E_TIMEOUT, MP_E_DIVERGED, or MP_E_NOT_CONVERGED (budget spent above tol)
};

// One stage of Algorithm 2's loop for increment s on cell c: exactly `target`
// iterations when target >= 0, else iterations until err <= tol, a failure,
// `budget` iterations, or (stag > 0) a stall of the error (stall_step with
// window stag, widening when adapt; gap: the longest gap between lows, carried
// between the increment's stages).  it0: iterations of the increment before
// the stage (trace numbering).  The loop runs on the device
// (one graph launch) unless a prescribed count, per-kernel timing or the
// trace needs the host between iterations.
template <class R>
mp_status run_loop(mp_rve* r, CellDev<R>& c, int s, cudaStream_t st, int target, int budget, int stag, bool adapt,
                   int& gap, int it0, LoopOut& o) {
  mp_ctx* ctx = r->ctx;
  o = LoopOut{};
  bool fused = false;
  if constexpr (sizeof(R) == 4) fused = r->use_fused && r->ctl.ptr != nullptr;
  auto count = [&](int n) {
    if (fused) {
      r->launches[MP_KC_SPECTRAL] += n;
    } else {
      if (c.n2 > 1) {
        r->launches[MP_KC_FFT_Y_FWD] += n;
        r->launches[MP_KC_FFT_Y_INV] += n;
      }
      r->launches[MP_KC_GREEN_Z] += n;
    }
    r->launches[MP_KC_PASS_A] += n;
    r->launches[MP_KC_REDUCE] += n;
  };
  auto classify = [&](const double* e) {
    if (e[5] != 0.0) o.status = MP_E_TIMEOUT;
    else if (!std::isfinite(e[0]) || e[0] > r->div_limit) o.status = MP_E_DIVERGED;
  };
  if (budget <= 0) {
    o.status = MP_E_NOT_CONVERGED;
    o.err = 2.0 * r->tol;
    return MP_OK;
  }
  if (target < 0 && !r->profiling && !r->tracing && r->device_loop) {
    r->loop_budget = budget;
    r->loop_stag = stag;
    r->loop_adapt = adapt ? 1 : 0;
    r->err_host[10] = (double)gap;
    const cudaError_t e = device_loop<R>(r, c, st, o.it, r->err_host);
    if (e == cudaErrorNotSupported) {
      r->device_loop = false;  // the host decides from now on
    } else {
      MP_CK(ctx, e);
      count(o.it);
      gap = (int)r->err_host[10];
      o.err = r->err_host[0];
      classify(r->err_host);
      if (o.status == MP_OK) {
        if (r->err_host[9] != 0.0) o.stalled = true;
        else if (o.err > r->tol) o.status = MP_E_NOT_CONVERGED;
      }
      return MP_OK;
    }
  }
  double err = 2.0 * r->tol, ref_err = 0.0;
  int it_ref = 0;
  const LaunchCfg& L = cfg_of<R>(r);
  double* parts = partials_of<R>(r);
  double* eout = reinterpret_cast<double*>(r->errout.ptr);
  const bool prof = r->profiling;
  auto mark = [&](int k, int end) {
    if (prof) cudaEventRecord(r->ev[2 * k + end], st);
  };
  while (target >= 0 ? o.it < target : err > r->tol) {
    if (target < 0 && o.it >= budget) {
      o.status = MP_E_NOT_CONVERGED;
      break;
    }
    if (fused) {
      if constexpr (sizeof(R) == 4) {
        mark(MP_KC_SPECTRAL, 0);
        MP_CK(ctx, launch_spectral(c, reinterpret_cast<int*>(r->ctl.ptr), ctx->nsm, st));
        mark(MP_KC_SPECTRAL, 1);
      }
    } else {
      mark(MP_KC_FFT_Y_FWD, 0);
      MP_CK(ctx, launch_fft_y<R>(L, c, -1, st));
      mark(MP_KC_FFT_Y_FWD, 1);
      mark(MP_KC_GREEN_Z, 0);
      MP_CK(ctx, launch_green_z<R>(L, c, st));
      mark(MP_KC_GREEN_Z, 1);
      mark(MP_KC_FFT_Y_INV, 0);
      MP_CK(ctx, launch_fft_y<R>(L, c, +1, st));
      mark(MP_KC_FFT_Y_INV, 1);
    }
    mark(MP_KC_PASS_A, 0);
    MP_CK(ctx, launch_pass_a_iter<R>(L, c, parts, st));
    mark(MP_KC_PASS_A, 1);
    mark(MP_KC_REDUCE, 0);
    MP_CK(ctx, launch_reduce_err<R>(L, c, parts, r->err_kind, eout, st));
    mark(MP_KC_REDUCE, 1);
    MP_CK(ctx, cudaMemcpyAsync(r->err_host, r->errout.ptr, sizeof(double) * 6, cudaMemcpyDeviceToHost, st));
    MP_CK(ctx, cudaStreamSynchronize(st));
    count(1);
    if (prof) {
      const int ks[6] = {MP_KC_FFT_Y_FWD, MP_KC_GREEN_Z, MP_KC_FFT_Y_INV, MP_KC_PASS_A, MP_KC_REDUCE,
                         MP_KC_SPECTRAL};
      for (int k : ks) {
        if (fused ? (k <= MP_KC_FFT_Y_INV) : (k == MP_KC_SPECTRAL)) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r->ev[2 * k], r->ev[2 * k + 1]) == cudaSuccess) r->kernel_ms[k] += ms;
      }
    }
    err = r->err_host[0];
    o.it += 1;
    o.err = err;
    if (r->tracing) {
      const double rec[7] = {(double)s, (double)(it0 + o.it), r->err_host[0], r->err_host[1], r->err_host[2],
                             r->err_host[3], r->err_host[4]};
      r->trace.insert(r->trace.end(), rec, rec + 7);
    }
    classify(r->err_host);
    if (o.status != MP_OK) break;
    // the stagnation watch, as on the device
    if (target < 0 && stag > 0 && err > r->tol && o.it < budget &&
        stall_step(err, o.it, stag, adapt, ref_err, it_ref, gap)) {
      o.stalled = true;
      break;
    }
  }
  return MP_OK;
}

// Moves the state of an FP32-mixed cell in the middle of increment s to its
// FP64 copy (records and predictor widened on the device; p, q and the cell
// scalars are shared; the polarization is formed anew there).
mp_status escalate_to_fp64(mp_rve* r, cudaStream_t st) {
  mp_ctx* ctx = r->ctx;
  mp_status s = twin_setup(r, st);
  if (s != MP_OK) return s;
  const long long nv = r->nvox;
  const int nsm = ctx->nsm;
  const CellDev<float>& f = r->cf;
  CellDev<double>& d = r->cd;
  MP_CK(ctx, (launch_convert<float, double>(f.prev, d.prev, 20 * nv, nsm, st)));
  MP_CK(ctx, (launch_convert<float, double>(f.hist, d.hist, 20 * nv, nsm, st)));
  MP_CK(ctx, (launch_convert<float, double>(f.elast, d.elast, 18 * nv, nsm, st)));
  return MP_OK;
}

// Back to FP32 after an increment committed in FP64 (the next increment's
// predictor is in the iterate record).
mp_status demote_from_fp64(mp_rve* r, cudaStream_t st) {
  mp_ctx* ctx = r->ctx;
  const long long nv = r->nvox;
  const int nsm = ctx->nsm;
  const CellDev<double>& d = r->cd;
  CellDev<float>& f = r->cf;
  MP_CK(ctx, (launch_convert<double, float>(d.prev, f.prev, 20 * nv, nsm, st)));
  MP_CK(ctx, (launch_convert<double, float>(d.hist, f.hist, 20 * nv, nsm, st)));
  MP_CK(ctx, (launch_convert<double, float>(d.elast, f.elast, 18 * nv, nsm, st)));
  return MP_OK;
}

// One load increment s (1-based): predictor, fixed-point loop, commit.
// An FP32-mixed cell (precision 1, no prescribed schedule, no manufactured
// source) whose error sets no new low in kStallIters iterations while above
// the tolerance continues the increment in the increment form (the first
// iteration writes tau(e^i) - tau(e^{i-1}), the next ones also transform the
// change of e); if that sets no new low in kStallItersDelta iterations (or
// twice the longest gap between the increment's earlier lows), the
// increment finishes in FP64 in the full form (restarted from the current
// iterate), is committed there and the state returns to FP32 for the next
// increment.
template <class R>
mp_status run_step(mp_rve* r, int s, cudaStream_t st) {
  mp_ctx* ctx = r->ctx;
  CellDev<R>& c = cell_of<R>(r);
  set_load(c, r, s);
  c.src = r->src.ptr ? reinterpret_cast<const R*>(r->src.ptr) + (size_t)(s - 1) * (size_t)r->nvox * 18 : nullptr;
  c.delta_in = c.delta_out = 0;
  const bool prof_step = r->profiling;
  if (prof_step) cudaEventRecord(r->ev[2 * MP_KC_START], st);
  MP_CK(ctx, launch_start<R>(r->L, c, s == 1 ? 1 : 0, st));
  if (prof_step) cudaEventRecord(r->ev[2 * MP_KC_START + 1], st);
  r->launches[MP_KC_START] += (s == 1) ? 2 : 1;
  const int target = r->lockstep.empty() ? -1 : r->lockstep[s - 1];
  const bool watch = sizeof(R) == 4 && r->precision == 1 && target < 0 && !r->src.ptr;
  LoopOut o;
  int it = 0, it64 = 0, gap = 0;
  bool in_fp64 = false;
  MP_CK_ST(run_loop<R>(r, c, s, st, target, target >= 0 ? target : r->max_iter, watch ? kStallIters : 0, false, gap,
                       0, o));
  it += o.it;
  if constexpr (sizeof(R) == 4) {
    if (o.stalled && !r->skip_delta) {
      // the increment form: one iteration that writes the first increment of
      // the polarization, then iterations on the increments
      ++r->delta_switches;
      c.delta_in = 0;
      c.delta_out = 1;
      if (it < r->max_iter) {
        MP_CK_ST(run_loop<R>(r, c, s, st, 1, 1, 0, false, gap, it, o));  // exactly one iteration
        it += o.it;
      } else {
        o.stalled = false;
        o.status = MP_E_NOT_CONVERGED;
      }
      if (o.status == MP_OK && o.err > r->tol) {
        c.delta_in = 1;
        MP_CK_ST(run_loop<R>(r, c, s, st, -1, r->max_iter - it, kStallItersDelta, true, gap, it, o));
        it += o.it;
      }
      if (o.stalled) r->skip_delta = true;  // it stalled here too: later stalls skip it
    }
    if (o.stalled) {
      ++r->escalations;
      MP_CK_ST(escalate_to_fp64(r, st));
      CellDev<double>& d = r->cd;
      set_load(d, r, s);
      d.src = nullptr;
      // FP64 restarts the full form from the current iterate: the start
      // pass forms its polarization, so the rounding the increment form
      // carried is damped by the iteration instead of kept
      d.delta_in = 0;
      d.delta_out = 0;
      MP_CK(ctx, launch_start<double>(r->L64, d, 0, st));
      r->launches[MP_KC_START] += 1;
      MP_CK_ST(run_loop<double>(r, d, s, st, -1, r->max_iter - it, 0, false, gap, it, o));
      it += o.it;
      it64 = o.it;
      in_fp64 = true;
    }
    c.delta_in = c.delta_out = 0;
  }
  const double err = o.err;
  mp_status status = o.status;
  if (status == MP_OK && o.stalled) status = MP_E_NOT_CONVERGED;  // a stall with no later stage
  r->total_iters += it;
  if (status == MP_E_TIMEOUT) {
    r->failed_step = s;
    r->steps_done = s - 1;
    return set_error(ctx, status, "load increment %d: a bounded device wait expired", s);
  }
  const bool predict = (status == MP_OK) && (s < r->n_steps);
  const double ratio =
      predict ? (r->time[s + 1] - r->time[s]) / (r->time[s] - r->time[s - 1]) : 0.0;
  double* row = reinterpret_cast<double*>(r->steprows.ptr) + (size_t)kAvgPartials * (s - 1);
  if (prof_step) cudaEventRecord(r->ev[2 * MP_KC_COMMIT], st);
  if (in_fp64) {
    CellDev<double>& d = r->cd;
    d.predict = predict ? 1 : 0;
    d.ratio = ratio;
    d.delta_in = d.delta_out = 0;
    MP_CK(ctx, launch_commit<double>(r->L64, d, avgpart_of<double>(r), row, st));
    MP_CK_ST(demote_from_fp64(r, st));
  } else {
    c.predict = predict ? 1 : 0;
    c.ratio = ratio;
    MP_CK(ctx, launch_commit<R>(r->L, c, avgpart_of<R>(r), row, st));
  }
  r->launches[MP_KC_COMMIT] += 2;
  if (prof_step) {
    // once per increment: the start and commit launches' times (the commit
    // class covers the commit and its averaging launch)
    MP_CK(ctx, cudaEventRecord(r->ev[2 * MP_KC_COMMIT + 1], st));
    MP_CK(ctx, cudaEventSynchronize(r->ev[2 * MP_KC_COMMIT + 1]));
    for (int k : {MP_KC_START, MP_KC_COMMIT}) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r->ev[2 * k], r->ev[2 * k + 1]) == cudaSuccess) r->kernel_ms[k] += ms;
    }
  }
  r->err_steps.push_back(err);
  r->iters_steps.push_back(it);
  r->iters64_steps.push_back(r->precision == 0 ? it : it64);
  r->steps_done = s;
  r->predicted = predict;
  if (status != MP_OK) {
    r->failed_step = s;
    return set_error(ctx, status, "load increment %d %s after %d iterations (err %.3e)", s,
                     status == MP_E_DIVERGED ? "diverged" : "did not converge", it, err);
  }
  return MP_OK;
}

// FNV-1a (64-bit) over the bytes that define a cell's problem: a checkpoint
// records it and a resume refuses another problem.
struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 1099511628211ull;
    }
  }
};

uint64_t problem_digest(const mp_problem* p, const double ref[6]) {
  Fnv f;
  f.add(p->n, sizeof(p->n));
  f.add(&p->h, sizeof(p->h));
  f.add(&p->precision, sizeof(p->precision));
  const long long nvox = (long long)p->n[0] * p->n[1] * p->n[2];
  f.add(p->phase, sizeof(uint16_t) * (size_t)nvox);
  f.add(p->phases, sizeof(mp_phase) * (size_t)p->n_phases);
  f.add(&p->n_steps, sizeof(p->n_steps));
  f.add(p->time, sizeof(double) * (size_t)(p->n_steps + 1));
  f.add(p->E, sizeof(double) * 9 * (size_t)(p->n_steps + 1));
  f.add(p->G, sizeof(double) * 9 * (size_t)(p->n_steps + 1));
  f.add(&p->tol, sizeof(p->tol));
  f.add(&p->err_kind, sizeof(p->err_kind));
  f.add(ref, sizeof(double) * 6);
  if (p->tau_m) {
    const size_t nsrc = (size_t)(p->n_steps + 1) * (size_t)nvox * 9;
    f.add(p->tau_m, sizeof(double) * nsrc);
    f.add(p->mu_m, sizeof(double) * nsrc);
  }
  return f.h;
}

// Checkpoint image: header, then the device arrays in this order.
struct CkptHeader {
  char magic[8];  // "MPCKPT2\0"
  int32_t precision, n[3], n_steps, steps_done, predicted, failed_step, skip_delta, reserved;
  int64_t total_iters;
  uint64_t digest;
  uint64_t bytes_prev, bytes_hist, bytes_pq, bytes_elast, bytes_tmean, bytes_rows;
};

void rve_free(mp_rve* r) {
  mp_ctx* ctx = r->ctx;
  DevBuf* bufs[] = {&r->spec, &r->prev, &r->hist, &r->pq, &r->elast, &r->phase, &r->phases,
                    &r->twx, &r->twy, &r->twz, &r->partials, &r->avgpart, &r->errout, &r->steprows,
                    &r->status, &r->tmean, &r->ctl, &r->src, &r->spec64, &r->prev64, &r->hist64,
                    &r->elast64, &r->phases64, &r->twx64, &r->twy64, &r->twz64, &r->partials64,
                    &r->avgpart64};
  for (DevBuf* b : bufs) dfree(ctx, *b);
  if (r->err_host) cudaFreeHost(r->err_host);
  r->err_host = nullptr;
  if (r->capture) cudaStreamDestroy(r->capture);
  r->capture = nullptr;
  for (auto& e : r->ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
}

}  // namespace

// ================================================================== C ABI
extern "C" {

int32_t mp_abi_version(void) { return MP_ABI_VERSION; }

const char* mp_last_error(const mp_ctx* ctx) {
  return ctx ? ctx->last_error.c_str() : last_error_global();
}

mp_status mp_validate(const mp_problem* problem, char* message, size_t message_len) {
  std::string msg;
  double ref[6];
  mp_status st = validate_problem(problem, nullptr, ref, msg);
  if (message && message_len > 0) {
    std::snprintf(message, message_len, "%s", msg.c_str());
  }
  return st;
}

mp_status mp_create(mp_ctx** out, int32_t device, const mp_alloc* alloc) {
  if (!out) return set_error(nullptr, MP_E_INVALID_ARG, "ctx pointer is NULL");
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count <= 0)
    return set_error(nullptr, MP_E_NO_DEVICE, "no CUDA device: %s", cudaGetErrorString(e));
  if (device < 0 || device >= count)
    return set_error(nullptr, MP_E_NO_DEVICE, "device %d out of range (%d devices)", device, count);
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return set_error(nullptr, MP_E_NO_DEVICE, "%s", cudaGetErrorString(e));
  mp_ctx* ctx = new mp_ctx();
  ctx->device = device;
  ctx->nsm = prop.multiProcessorCount;
  if (alloc && alloc->alloc && alloc->free) {
    ctx->alloc = *alloc;
    ctx->has_alloc = true;
  }
  *out = ctx;
  return MP_OK;
}

void mp_destroy(mp_ctx* ctx) { delete ctx; }

mp_status mp_rve_create(mp_ctx* ctx, const mp_problem* p, mp_rve** out, void* stream) {
  if (!ctx || !out) return set_error(ctx, MP_E_INVALID_ARG, "NULL argument");
  *out = nullptr;
  std::string msg;
  double ref[6];
  std::vector<long long> counts;
  mp_status st = validate_problem(p, &counts, ref, msg);
  if (st != MP_OK) return set_error(ctx, st, "%s", msg.c_str());
  MP_DEVICE_SCOPE(ctx);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  mp_rve* r = new mp_rve();
  r->ctx = ctx;
  r->precision = p->precision;
  for (int j = 0; j < 3; ++j) r->n[j] = p->n[j];
  r->nvox = (long long)p->n[0] * p->n[1] * p->n[2];
  r->h = p->h;
  r->n_steps = p->n_steps;
  r->time.assign(p->time, p->time + p->n_steps + 1);
  r->E.assign(p->E, p->E + 9 * (p->n_steps + 1));
  r->G.assign(p->G, p->G + 9 * (p->n_steps + 1));
  r->tol = p->tol;
  r->err_kind = p->err_kind;
  r->max_iter = p->max_iter > 0 ? p->max_iter : 10000;
  if (p->lockstep_iters) r->lockstep.assign(p->lockstep_iters, p->lockstep_iters + p->n_steps);
  r->div_limit = p->div_limit > 0 ? p->div_limit : 1e6;
  for (int i = 0; i < 6; ++i) r->ref[i] = ref[i];
  cudaError_t e = cudaMallocHost(&r->err_host, sizeof(double) * 16);
  if (e != cudaSuccess) {
    r->err_host = nullptr;
    delete r;
    return set_error(ctx, MP_E_CUDA, "cudaMallocHost: %s", cudaGetErrorString(e));
  }
  for (int i = 0; i < 16; ++i) r->err_host[i] = 0.0;
  r->phases_host.assign(p->phases, p->phases + p->n_phases);
  r->digest = problem_digest(p, ref);
  st = (r->precision == 0) ? rve_setup<double>(r, p, cs) : rve_setup<float>(r, p, cs);
  if (st == MP_OK && ctx->autotune)
    st = (r->precision == 0) ? rve_autotune<double>(r, cs) : rve_autotune<float>(r, cs);
  if (st != MP_OK) {
    rve_free(r);
    delete r;
    return st;
  }
  *out = r;
  return MP_OK;
}

mp_status mp_rve_reset(mp_rve* r, void* stream) {
  if (!r) return set_error(nullptr, MP_E_INVALID_ARG, "rve is NULL");
  MP_DEVICE_SCOPE(r->ctx);
  mp_status st = MP_OK;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  // the transform constants start from zero as in a fresh cell
  MP_CK(r->ctx, cudaMemsetAsync(r->tmean.ptr, 0, r->tmean.bytes, cs));
  MP_CK(r->ctx, cudaMemsetAsync(r->status.ptr, 0, r->status.bytes, cs));
  r->steps_done = 0;
  r->predicted = false;
  r->total_iters = 0;
  r->failed_step = 0;
  r->err_steps.clear();
  r->iters_steps.clear();
  r->iters64_steps.clear();
  r->skip_delta = false;
  return MP_OK;
}

mp_status mp_checkpoint(mp_rve* r, void* host_buf, size_t* bytes, void* stream) {
  if (!r || !bytes) return set_error(r ? r->ctx : nullptr, MP_E_INVALID_ARG, "NULL argument");
  CkptHeader h{};
  std::memcpy(h.magic, "MPCKPT2", 8);
  h.precision = r->precision;
  for (int j = 0; j < 3; ++j) h.n[j] = r->n[j];
  h.n_steps = r->n_steps;
  h.steps_done = r->steps_done;
  h.predicted = r->predicted ? 1 : 0;
  h.failed_step = r->failed_step;
  h.skip_delta = r->skip_delta ? 1 : 0;
  h.total_iters = r->total_iters;
  h.digest = r->digest;
  h.bytes_prev = r->prev.bytes;
  h.bytes_hist = r->hist.bytes;
  h.bytes_pq = r->pq.bytes;
  h.bytes_elast = r->elast.bytes;
  h.bytes_tmean = r->tmean.bytes;
  h.bytes_rows = r->steprows.bytes;
  const size_t host_bytes = sizeof(double) * r->err_steps.size() + 2 * sizeof(int32_t) * r->iters_steps.size();
  const size_t need = sizeof(h) + h.bytes_prev + h.bytes_hist + h.bytes_pq + h.bytes_elast + h.bytes_tmean +
                      h.bytes_rows + host_bytes;
  if (!host_buf) {
    *bytes = need;
    return MP_OK;
  }
  if (*bytes < need) {
    *bytes = need;
    return set_error(r->ctx, MP_E_INVALID_ARG, "checkpoint buffer too small (%zu bytes needed)", need);
  }
  MP_DEVICE_SCOPE(r->ctx);
  mp_status st = MP_OK;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  unsigned char* out = static_cast<unsigned char*>(host_buf);
  std::memcpy(out, &h, sizeof(h));
  size_t o = sizeof(h);
  const DevBuf* arrs[6] = {&r->prev, &r->hist, &r->pq, &r->elast, &r->tmean, &r->steprows};
  for (const DevBuf* b : arrs) {
    MP_CK(r->ctx, cudaMemcpyAsync(out + o, b->ptr, b->bytes, cudaMemcpyDeviceToHost, cs));
    o += b->bytes;
  }
  MP_CK(r->ctx, cudaStreamSynchronize(cs));
  for (size_t k = 0; k < r->err_steps.size(); ++k) {
    std::memcpy(out + o, &r->err_steps[k], sizeof(double));
    o += sizeof(double);
  }
  for (size_t k = 0; k < r->iters_steps.size(); ++k) {
    const int32_t it = r->iters_steps[k];
    std::memcpy(out + o, &it, sizeof(int32_t));
    o += sizeof(int32_t);
  }
  for (size_t k = 0; k < r->iters64_steps.size(); ++k) {
    const int32_t it = r->iters64_steps[k];
    std::memcpy(out + o, &it, sizeof(int32_t));
    o += sizeof(int32_t);
  }
  *bytes = o;
  return MP_OK;
}

mp_status mp_resume(mp_rve* r, const void* host_buf, size_t bytes, void* stream) {
  if (!r || !host_buf) return set_error(r ? r->ctx : nullptr, MP_E_INVALID_ARG, "NULL argument");
  CkptHeader h;
  if (bytes < sizeof(h)) return set_error(r->ctx, MP_E_INVALID_ARG, "checkpoint truncated");
  std::memcpy(&h, host_buf, sizeof(h));
  if (std::memcmp(h.magic, "MPCKPT2", 8) != 0)
    return set_error(r->ctx, MP_E_INVALID_ARG, "not a checkpoint of this library");
  if (h.digest != r->digest || h.precision != r->precision || h.n_steps != r->n_steps ||
      h.n[0] != r->n[0] || h.n[1] != r->n[1] || h.n[2] != r->n[2])
    return set_error(r->ctx, MP_E_INVALID_ARG, "checkpoint belongs to another problem or precision");
  if (h.bytes_prev != r->prev.bytes || h.bytes_hist != r->hist.bytes || h.bytes_pq != r->pq.bytes ||
      h.bytes_elast != r->elast.bytes || h.bytes_tmean != r->tmean.bytes || h.bytes_rows != r->steprows.bytes ||
      h.steps_done < 0 || h.steps_done > r->n_steps)
    return set_error(r->ctx, MP_E_INVALID_ARG, "checkpoint layout does not match the cell");
  const size_t nst = (size_t)h.steps_done;
  const size_t need = sizeof(h) + h.bytes_prev + h.bytes_hist + h.bytes_pq + h.bytes_elast + h.bytes_tmean +
                      h.bytes_rows + nst * (sizeof(double) + 2 * sizeof(int32_t));
  if (bytes < need) return set_error(r->ctx, MP_E_INVALID_ARG, "checkpoint truncated");
  MP_DEVICE_SCOPE(r->ctx);
  mp_status st = MP_OK;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  const unsigned char* in = static_cast<const unsigned char*>(host_buf);
  size_t o = sizeof(h);
  DevBuf* arrs[6] = {&r->prev, &r->hist, &r->pq, &r->elast, &r->tmean, &r->steprows};
  for (DevBuf* b : arrs) {
    MP_CK(r->ctx, cudaMemcpyAsync(b->ptr, in + o, b->bytes, cudaMemcpyHostToDevice, cs));
    o += b->bytes;
  }
  MP_CK(r->ctx, cudaMemsetAsync(r->status.ptr, 0, r->status.bytes, cs));
  MP_CK(r->ctx, cudaStreamSynchronize(cs));
  r->err_steps.assign(nst, 0.0);
  r->iters_steps.assign(nst, 0);
  for (size_t k = 0; k < nst; ++k) {
    std::memcpy(&r->err_steps[k], in + o, sizeof(double));
    o += sizeof(double);
  }
  for (size_t k = 0; k < nst; ++k) {
    int32_t it;
    std::memcpy(&it, in + o, sizeof(int32_t));
    r->iters_steps[k] = it;
    o += sizeof(int32_t);
  }
  r->iters64_steps.assign(nst, 0);
  for (size_t k = 0; k < nst; ++k) {
    int32_t it;
    std::memcpy(&it, in + o, sizeof(int32_t));
    r->iters64_steps[k] = it;
    o += sizeof(int32_t);
  }
  r->steps_done = h.steps_done;
  r->predicted = h.predicted != 0;
  r->failed_step = h.failed_step;
  r->skip_delta = h.skip_delta != 0;
  r->total_iters = h.total_iters;
  return MP_OK;
}

mp_status mp_rve_run(mp_rve* r, int32_t n_steps, void* stream) {
  if (!r) return set_error(nullptr, MP_E_INVALID_ARG, "rve is NULL");
  MP_DEVICE_SCOPE(r->ctx);
  mp_status st = MP_OK;
  if (r->failed_step) return set_error(r->ctx, MP_E_INVALID_ARG, "cell failed at step %d; reset first", r->failed_step);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  for (int k = 0; k < n_steps && r->steps_done < r->n_steps; ++k) {
    const int s = r->steps_done + 1;
    st = (r->precision == 0) ? run_step<double>(r, s, cs) : run_step<float>(r, s, cs);
    if (st != MP_OK) return st;
  }
  return MP_OK;
}

int32_t mp_rve_steps_done(const mp_rve* r) { return r ? r->steps_done : 0; }

mp_status mp_set_autotune(mp_ctx* ctx, int32_t enable) {
  if (!ctx) return set_error(nullptr, MP_E_INVALID_ARG, "ctx is NULL");
  ctx->autotune = enable != 0;
  return MP_OK;
}

mp_status mp_rve_config(const mp_rve* r, int32_t* cfg, int32_t n) {
  if (!r || !cfg || n < 0) return set_error(nullptr, MP_E_INVALID_ARG, "NULL argument");
  bool fused = r->use_fused && r->ctl.ptr != nullptr;
  const int32_t v[6] = {r->L.rows, fused ? 1 : 0, r->L.grid_a, r->L.grid_y, r->L.grid_z, r->tuned ? 1 : 0};
  for (int i = 0; i < n && i < 6; ++i) cfg[i] = v[i];
  return MP_OK;
}

mp_status mp_rve_profile(mp_rve* r, int32_t enable) {
  if (!r) return set_error(nullptr, MP_E_INVALID_ARG, "rve is NULL");
  MP_DEVICE_SCOPE(r->ctx);
  mp_status st = MP_OK;
  if (enable && !r->ev[0]) {
    for (auto& e : r->ev) MP_CK(r->ctx, cudaEventCreate(&e));
  }
  r->profiling = enable != 0;
  return MP_OK;
}

mp_status mp_rve_trace(mp_rve* r, int32_t enable) {
  if (!r) return set_error(nullptr, MP_E_INVALID_ARG, "rve is NULL");
  r->tracing = enable != 0;
  if (!r->tracing) r->trace.clear();
  return MP_OK;
}

int64_t mp_rve_trace_read(mp_rve* r, double* out, int64_t capacity, int32_t clear) {
  if (!r) return -1;
  const int64_t n = (int64_t)(r->trace.size() / 7);
  if (out) {
    const int64_t k = n < capacity ? n : capacity;
    std::memcpy(out, r->trace.data(), sizeof(double) * 7 * (size_t)k);
  }
  if (clear) r->trace.clear();
  return n;
}

mp_status mp_rve_profile_read(const mp_rve* r, double* ms, int64_t* launches, int32_t reset) {
  if (!r) return set_error(nullptr, MP_E_INVALID_ARG, "rve is NULL");
  for (int k = 0; k < MP_KC_COUNT; ++k) {
    if (ms) ms[k] = r->kernel_ms[k];
    if (launches) launches[k] = r->launches[k];
  }
  if (reset) {
    mp_rve* w = const_cast<mp_rve*>(r);
    for (int k = 0; k < MP_KC_COUNT; ++k) {
      w->kernel_ms[k] = 0.0;
      w->launches[k] = 0;
    }
  }
  return MP_OK;
}
int64_t mp_rve_iterations(const mp_rve* r) { return r ? r->total_iters : 0; }

mp_status mp_rve_results(mp_rve* r, mp_result* res, void* stream) {
  if (!r || !res) return set_error(r ? r->ctx : nullptr, MP_E_INVALID_ARG, "NULL argument");
  mp_ctx* ctx = r->ctx;
  MP_DEVICE_SCOPE(ctx);
  mp_status st = MP_OK;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  const int ns = r->steps_done;
  std::vector<double> rows((size_t)kAvgPartials * (ns > 0 ? ns : 1));
  if (ns > 0)
    MP_CK(ctx, cudaMemcpyAsync(rows.data(), r->steprows.ptr, sizeof(double) * kAvgPartials * ns,
                               cudaMemcpyDeviceToHost, cs));
  // final fields (of the last committed step)
  const bool want = res->e || res->g || res->t || res->m || res->p || res->q;
  DevBuf fbuf;
  if (want && ns > 0) {
    const size_t nv = (size_t)r->nvox;
    if ((st = dalloc(ctx, fbuf, sizeof(double) * 38 * nv)) != MP_OK) return st;
    double* b = reinterpret_cast<double*>(fbuf.ptr);
    double *fe = b, *fg = b + 9 * nv, *ft = b + 18 * nv, *fm = b + 27 * nv, *fp = b + 36 * nv, *fq = b + 37 * nv;
    cudaError_t e = (r->precision == 0)
                        ? launch_fields<double>(r->L, r->cd, r->predicted ? 1 : 0, fe, fg, ft, fm, fp, fq, cs)
                        : launch_fields<float>(r->L, r->cf, r->predicted ? 1 : 0, fe, fg, ft, fm, fp, fq, cs);
    if (e != cudaSuccess) {
      dfree(ctx, fbuf);
      return set_error(ctx, MP_E_CUDA, "fields kernel: %s", cudaGetErrorString(e));
    }
    struct {
      double* dst;
      double* src;
      size_t n;
    } cp[6] = {{res->e, fe, 9 * nv}, {res->g, fg, 9 * nv}, {res->t, ft, 9 * nv},
               {res->m, fm, 9 * nv}, {res->p, fp, nv},     {res->q, fq, nv}};
    for (auto& x : cp)
      if (x.dst) {
        e = cudaMemcpyAsync(x.dst, x.src, sizeof(double) * x.n, cudaMemcpyDeviceToHost, cs);
        if (e != cudaSuccess) break;
      }
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    dfree(ctx, fbuf);
    if (e != cudaSuccess) return set_error(ctx, MP_E_CUDA, "field copy: %s", cudaGetErrorString(e));
  }
  MP_CK(ctx, cudaStreamSynchronize(cs));
  for (int s = 0; s < ns; ++s) {
    const double* row = rows.data() + (size_t)kAvgPartials * s;
    for (int q = 0; q < 9; ++q) {
      if (res->T) res->T[9 * s + q] = row[q];
      if (res->M) res->M[9 * s + q] = row[9 + q];
      if (res->Eavg) res->Eavg[9 * s + q] = row[18 + q];
      if (res->Gavg) res->Gavg[9 * s + q] = row[27 + q];
    }
    if (res->P) res->P[s] = row[36];
    if (res->Q) res->Q[s] = row[37];
    if (res->Teq) res->Teq[s] = row[38];
    if (res->Meq) res->Meq[s] = row[39];
    if (res->err) res->err[s] = r->err_steps[s];
    if (res->iters) res->iters[s] = r->iters_steps[s];
    if (res->iters_fp64) res->iters_fp64[s] = r->iters64_steps[s];
  }
  res->steps_done = ns;
  res->failed_step = r->failed_step;
  for (int i = 0; i < 6; ++i) res->ref_moduli_used[i] = r->ref[i];
  return MP_OK;
}

void mp_rve_destroy(mp_rve* r) {
  if (!r) return;
  if (r->ctx) {
    DeviceScope dev(r->ctx->device);
    rve_free(r);
  } else {
    rve_free(r);
  }
  delete r;
}

mp_status mp_solve(mp_ctx* ctx, const mp_problem* p, mp_result* res, void* stream) {
  mp_rve* r = nullptr;
  mp_status st = mp_rve_create(ctx, p, &r, stream);
  if (st != MP_OK) return st;
  mp_status run = mp_rve_run(r, p->n_steps, stream);
  std::string run_msg = ctx->last_error;
  if (res) {
    mp_status rs = mp_rve_results(r, res, stream);
    if (run == MP_OK && rs != MP_OK) run = rs;
  }
  mp_rve_destroy(r);
  if (run != MP_OK && !run_msg.empty()) ctx->last_error = run_msg;
  return run;
}

// ------------------------------------------------------------------ components
mp_status mp_radial_return(mp_ctx* ctx, int32_t precision, int64_t count, const uint16_t* phase,
                           int32_t n_phases, const mp_phase* phases, const void* e, const void* g,
                           const void* e_n, const void* g_n, const void* t_n, const void* m_n,
                           const double* p_n, const double* q_n, void* t, void* m, double* p,
                           double* q, void* stream) {
  if (!ctx) return set_error(nullptr, MP_E_INVALID_ARG, "ctx is NULL");
  if (count < 0 || n_phases < 1 || !phases || precision < 0 || precision > 2)
    return set_error(ctx, MP_E_INVALID_ARG, "invalid arguments");
  if (count > 0 && (!phase || !e || !g || !e_n || !g_n || !t_n || !m_n || !p_n || !q_n || !t || !m || !p || !q))
    return set_error(ctx, MP_E_INVALID_ARG, "NULL buffer");
  std::string msg;
  for (int k = 0; k < n_phases; ++k) {
    mp_status s = check_phase(phases[k], k, msg);
    if (s != MP_OK) return set_error(ctx, s, "%s", msg.c_str());
  }
  MP_DEVICE_SCOPE(ctx);
  mp_status st = MP_OK;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  DevBuf tab;
  if (precision == 0) {
    std::vector<PhaseDev<double>> ph(n_phases);
    for (int k = 0; k < n_phases; ++k) ph[k] = phase_dev<double>(phases[k]);
    if ((st = dalloc(ctx, tab, sizeof(PhaseDev<double>) * n_phases)) != MP_OK) return st;
    cudaError_t e1 = cudaMemcpyAsync(tab.ptr, ph.data(), tab.bytes, cudaMemcpyHostToDevice, cs);
    if (e1 == cudaSuccess)
      e1 = launch_radial_return<double>(ctx->nsm, count, phase, (const PhaseDev<double>*)tab.ptr,
                                        (const double*)e, (const double*)g, (const double*)e_n,
                                        (const double*)g_n, (const double*)t_n, (const double*)m_n, p_n,
                                        q_n, (double*)t, (double*)m, p, q, cs);
    if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(cs);
    dfree(ctx, tab);
    if (e1 != cudaSuccess) return set_error(ctx, MP_E_CUDA, "radial return: %s", cudaGetErrorString(e1));
  } else {
    std::vector<PhaseDev<float>> ph(n_phases);
    for (int k = 0; k < n_phases; ++k) ph[k] = phase_dev<float>(phases[k], precision == 2);
    if ((st = dalloc(ctx, tab, sizeof(PhaseDev<float>) * n_phases)) != MP_OK) return st;
    cudaError_t e1 = cudaMemcpyAsync(tab.ptr, ph.data(), tab.bytes, cudaMemcpyHostToDevice, cs);
    if (e1 == cudaSuccess)
      e1 = launch_radial_return<float>(ctx->nsm, count, phase, (const PhaseDev<float>*)tab.ptr,
                                       (const float*)e, (const float*)g, (const float*)e_n,
                                       (const float*)g_n, (const float*)t_n, (const float*)m_n, p_n,
                                       q_n, (float*)t, (float*)m, p, q, cs);
    if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(cs);
    dfree(ctx, tab);
    if (e1 != cudaSuccess) return set_error(ctx, MP_E_CUDA, "radial return: %s", cudaGetErrorString(e1));
  }
  return MP_OK;
}

}  // extern "C"

namespace {
template <class R>
mp_status green_apply_impl(mp_ctx* ctx, const int32_t n[3], double h, const double ref[6], const void* tau,
                           const void* mu, void* e_out, void* g_out, cudaStream_t cs) {
  CellDev<R> c{};
  c.n1 = n[0];
  c.n2 = n[1];
  c.n3 = n[2];
  c.kx = (c.n1 > 1) ? c.n1 / 2 : 1;
  c.nvox = (long long)n[0] * n[1] * n[2];
  c.nspec = (long long)c.kx * n[1] * n[2];
  c.h = h;
  c.inv_nvox = 1.0 / (double)c.nvox;
  for (int j = 0; j < 3; ++j) c.two_pi_over_L[j] = (R)(2.0 * M_PI / ((double)n[j] * h));
  c.ref = ref_dev<R>(ref);
  DevBuf spec, tx, ty, tz, stat, ctl;
  std::vector<cpx<R>> h1, h2, h3;
  mp_status st = dalloc(ctx, spec, sizeof(cpx<R>) * 18 * (size_t)c.nspec);
  if (st == MP_OK) st = dalloc(ctx, stat, sizeof(int) * 4);
  if (st == MP_OK && cudaMemsetAsync(stat.ptr, 0, stat.bytes, cs) != cudaSuccess)
    st = set_error(ctx, MP_E_CUDA, "cudaMemsetAsync failed");
  c.status = reinterpret_cast<int*>(stat.ptr);
  if (st == MP_OK) st = make_axis<R>(ctx, c.n1, true, c.px, tx, cs, h1);
  if (st == MP_OK) st = make_axis<R>(ctx, c.n2, false, c.py, ty, cs, h2);
  if (st == MP_OK) st = make_axis<R>(ctx, c.n3, false, c.pz, tz, cs, h3);
  if constexpr (sizeof(R) == 4) {
    if (st == MP_OK && spectral_fused_ok(c)) st = dalloc(ctx, ctl, sizeof(int) * spectral_ctl_ints(c.kx));
    if (st == MP_OK && ctl.ptr && cudaMemsetAsync(ctl.ptr, 0, ctl.bytes, cs) != cudaSuccess)
      st = set_error(ctx, MP_E_CUDA, "cudaMemsetAsync failed");
  }
  if (st == MP_OK) {
    c.spec = reinterpret_cast<cpx<R>*>(spec.ptr);
    LaunchCfg L = make_launch_cfg<R>(c, ctx->nsm);
    c.rows_a = L.rows;
    c.items_a = L.items_a;
    cudaError_t e = launch_green_apply<R>(L, c, (const R*)tau, (const R*)mu, (R*)e_out, (R*)g_out, cs,
                                          reinterpret_cast<int*>(ctl.ptr), ctx->nsm);
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, stat.ptr, sizeof(int), cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) st = set_error(ctx, MP_E_CUDA, "green apply: %s", cudaGetErrorString(e));
    else if (flag) st = set_error(ctx, MP_E_TIMEOUT, "green apply: a bounded device wait expired");
  }
  cudaStreamSynchronize(cs);
  dfree(ctx, spec);
  dfree(ctx, stat);
  dfree(ctx, tx);
  dfree(ctx, ty);
  dfree(ctx, tz);
  dfree(ctx, ctl);
  return st;
}
}  // namespace

extern "C" {

mp_status mp_green_apply(mp_ctx* ctx, int32_t precision, const int32_t n[3], double h,
                         const double ref_moduli[6], const void* tau, const void* mu, void* e_out,
                         void* g_out, void* stream) {
  if (!ctx) return set_error(nullptr, MP_E_INVALID_ARG, "ctx is NULL");
  if (!n || !ref_moduli || !tau || !mu || !e_out || !g_out || precision < 0 || precision > 2)
    return set_error(ctx, MP_E_INVALID_ARG, "invalid arguments");
  for (int j = 0; j < 3; ++j)
    if (n[j] < 1 || !size_ok(n[j])) return set_error(ctx, MP_E_UNSUPPORTED_SIZE, "grid size %d unsupported", n[j]);
  if (!(h > 0)) return set_error(ctx, MP_E_INVALID_ARG, "h must be positive");
  const double* r = ref_moduli;
  if (!(r[0] + 2 * r[1] > 0) || !(r[1] > 0) || !(r[2] > 0) || !(r[5] >= 0) || !(r[3] + r[4] + r[5] >= 0))
    return set_error(ctx, MP_E_INADMISSIBLE, "reference medium not admissible for the Green operator");
  MP_DEVICE_SCOPE(ctx);
  mp_status st = MP_OK;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  return precision == 0 ? green_apply_impl<double>(ctx, n, h, ref_moduli, tau, mu, e_out, g_out, cs)
                        : green_apply_impl<float>(ctx, n, h, ref_moduli, tau, mu, e_out, g_out, cs);
}

}  // extern "C"
