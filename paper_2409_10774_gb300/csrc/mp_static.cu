// mp_green_apply_static: the Green-operator application of mp_green_apply
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they need the operator: for example an application that hands this library
// a fixed device-memory budget reserved up front by another runtime, or a
// latency-critical loop that must not trigger the implicit device
// synchronisation and the out-of-memory failures that cudaMalloc / cudaFree
// can bring.  This entry point therefore works entirely in one file-scope
// device array, `g_static_scratch`, of MP_STATIC_SCRATCH_BYTES: its first
// 32 KiB hold the status word and the three twiddle tables, the rest holds
// the 18-component half spectrum.  Every GPU that loads the library holds
// this array until the process exits.
//
// The array's name is only a host-side stand-in in host code; its device
// address is looked up with cudaGetSymbolAddress once per device, with that
// device current, on the first call made on the device (make that first
// call before any stream capture).  A context is required (as for
// mp_green_apply): its device is made current for the call and the caller's
// current device is restored on return.  All calls share the array and it keeps
// the last call's contents: the status word is cleared on every call, and
// the spectrum is fully overwritten by the forward transform before it is
// read.  Calls whose work overlaps on the GPU (other streams, other host
// threads) race on the array; serialise them.
#include <cmath>
#include <mutex>

#include "../../include/micropolar.h"
#include "mp_host.cuh"
#include "mp_kernels.cuh"

using namespace mp;

namespace {

constexpr size_t kTableRegion = 32 * 1024;  // status word + three twiddle tables
constexpr size_t kSpectrumBytes = MP_STATIC_SCRATCH_BYTES - kTableRegion;
constexpr int kMaxAxis = 512;

static __device__ __align__(256) unsigned char g_static_scratch[MP_STATIC_SCRATCH_BYTES];

std::mutex g_setup_mutex;
void* g_scratch_ptr[64] = {nullptr};

mp_status fail(mp_ctx* ctx, mp_status st, const char* msg) { return set_error(ctx, st, "%s", msg); }

// Device address of the scratch array for the context's device, which the
// caller has made current (set-up on the first call made on that device).
mp_status scratch_for_device(mp_ctx* ctx, void** out) {
  const int dev = ctx->device;
  if (dev < 0 || dev >= 64) return fail(ctx, MP_E_NO_DEVICE, "mp_green_apply_static: device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return set_error(ctx, MP_E_CUDA, "mp_green_apply_static: cudaGetSymbolAddress failed: %s",
                       cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return MP_OK;
}

bool axis_ok(int n) {
  if (n == 1) return true;
  if (n < 2 || n > kMaxAxis || (n % 2) != 0) return false;
  while (n % 2 == 0) n /= 2;
  while (n % 3 == 0) n /= 3;
  return n == 1;
}

template <class R>
mp_status run(mp_ctx* ctx, const int32_t n[3], double h, const double ref[6], const void* tau,
              const void* mu, void* e_out, void* g_out, cudaStream_t st) {
  void* base = nullptr;
  mp_status s = scratch_for_device(ctx, &base);
  if (s != MP_OK) return s;
  unsigned char* b = static_cast<unsigned char*>(base);
  int* status = reinterpret_cast<int*>(b);
  cpx<R>* tw[3];
  for (int a = 0; a < 3; ++a) tw[a] = reinterpret_cast<cpx<R>*>(b + 256 + (size_t)a * kMaxAxis * sizeof(cpx<double>));

  CellDev<R> c{};
  c.n1 = n[0];
  c.n2 = n[1];
  c.n3 = n[2];
  c.kx = (c.n1 > 1) ? c.n1 / 2 : 1;
  c.nvox = (long long)n[0] * n[1] * n[2];
  c.nspec = (long long)c.kx * n[1] * n[2];
  if ((size_t)c.nspec * 18 * sizeof(cpx<R>) > kSpectrumBytes)
    return fail(ctx, MP_E_UNSUPPORTED_SIZE,
                "mp_green_apply_static: grid needs more than the static scratch array "
                "(18 complex values per half-spectrum point must fit in MP_STATIC_SCRATCH_BYTES - 32 KiB)");
  c.h = h;
  c.inv_nvox = 1.0 / (double)c.nvox;
  for (int j = 0; j < 3; ++j) c.two_pi_over_L[j] = (R)(2.0 * M_PI / ((double)n[j] * h));
  c.ref.lam = (R)ref[0];
  c.ref.mu = (R)ref[1];
  c.ref.kap = (R)ref[2];
  c.ref.alpha = (R)ref[3];
  c.ref.beta = (R)ref[4];
  c.ref.gamma = (R)ref[5];
  c.spec = reinterpret_cast<cpx<R>*>(b + kTableRegion);
  c.status = status;
  AxisPlan<R>* plans[3] = {&c.px, &c.py, &c.pz};
  // twiddle tables W_N^k = exp(-2 pi i k / N), built on the host stack and copied in
  static thread_local cpx<R> host_tw[3][kMaxAxis];
  for (int a = 0; a < 3; ++a) {
    axis_plan<R>(n[a], a == 0, *plans[a], host_tw[a]);  // the plans every entry point uses
    plans[a]->tw = tw[a];
  }
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  for (int a = 0; a < 3 && e == cudaSuccess; ++a)
    e = cudaMemcpyAsync(tw[a], host_tw[a], sizeof(cpx<R>) * n[a], cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    LaunchCfg L = make_launch_cfg<R>(c, ctx->nsm > 0 ? ctx->nsm : 1);
    c.rows_a = L.rows;
    c.items_a = L.items_a;
    e = launch_green_apply<R>(L, c, (const R*)tau, (const R*)mu, (R*)e_out, (R*)g_out, st);
  }
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(ctx, MP_E_CUDA, cudaGetErrorString(e));
  if (flag) return fail(ctx, MP_E_TIMEOUT, "mp_green_apply_static: a bounded device wait expired");
  return MP_OK;
}

}  // namespace

extern "C" {

mp_status mp_green_apply_static(mp_ctx* ctx, int32_t precision, const int32_t n[3], double h,
                                const double ref_moduli[6], const void* tau, const void* mu,
                                void* e_out, void* g_out, void* stream) {
  if (!ctx) return set_error(nullptr, MP_E_INVALID_ARG, "mp_green_apply_static: ctx is NULL");
  if (!n || !ref_moduli || !tau || !mu || !e_out || !g_out || precision < 0 || precision > 2)
    return fail(ctx, MP_E_INVALID_ARG, "mp_green_apply_static: invalid arguments");
  for (int j = 0; j < 3; ++j)
    if (!axis_ok(n[j]))
      return fail(ctx, MP_E_UNSUPPORTED_SIZE, "mp_green_apply_static: grid size unsupported");
  if (!(h > 0)) return fail(ctx, MP_E_INVALID_ARG, "mp_green_apply_static: h must be positive");
  const double* r = ref_moduli;
  if (!(r[0] + 2 * r[1] > 0) || !(r[1] > 0) || !(r[2] > 0) || !(r[5] >= 0) || !(r[3] + r[4] + r[5] >= 0))
    return fail(ctx, MP_E_INADMISSIBLE, "mp_green_apply_static: reference medium not admissible");
  if (!(precision == 0 ? sizes_fit<double>(n[0], n[1], n[2]) : sizes_fit<float>(n[0], n[1], n[2])))
    return fail(ctx, MP_E_UNSUPPORTED_SIZE, "mp_green_apply_static: grid too large for the tiles");
  MP_DEVICE_SCOPE(ctx);  // the context's device, the caller's given back on return
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return precision == 0 ? run<double>(ctx, n, h, ref_moduli, tau, mu, e_out, g_out, st)
                        : run<float>(ctx, n, h, ref_moduli, tau, mu, e_out, g_out, st);
}

}  // extern "C"
