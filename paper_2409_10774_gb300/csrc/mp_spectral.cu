// Fused spectral pass of one fixed-point iteration (sm_103a, FP32 fields):
// y forward, z forward, Green operator (eq. micropolar_LippmannSchwinger_iteration),
// z inverse and y inverse of the 18-component half spectrum, for cells whose
// y and z lengths are 256.
//
// The three separate column passes (y forward, z + Green + z, y inverse) each
// stream the whole 1.2 GB spectrum of a 256^3 cell through HBM.  Here one
// persistent kernel runs them as three phases per kx column-plane (all y and
// z of one kx: 256 x 256 points x 18 components, 9.4 MB in FP32) and takes
// its work items from one queue in the order
//     Y-forward(g), Z(g - 1), Y-inverse(g - 2),  g = 0, 1, 2, ...
// so that a plane is read from HBM by its Y-forward items, revisited by its Z
// and Y-inverse items while it is still in L2 (about three planes, 28 MB, are
// live at a time), and written back once.  A Z item of plane g waits until
// every Y-forward item of g has finished, a Y-inverse item until every Z item
// of g has; since items are taken in queue order and each waits only on
// items taken before it (held by running blocks), the waits always end.  They
// are bounded all the same: a wait that gives up records status bit 1 and the
// item is skipped (the host reports MP_E_TIMEOUT).
//
// Each item is one column of 18 lines x 256 points; its 288 threads are
// (line c, butterfly j), 18 x 16.  The 256-point transform is two radix-16
// Stockham stages: stage one from global memory into registers, a transpose
// through shared memory, stage two with the twiddles W_256^(r j), and the
// result back to global memory (the Z item keeps it in shared memory for the
// Green operator and the inverse transform).
#include "mp_fft.cuh"
#include "mp_green.cuh"
#include "mp_kernels.cuh"

namespace mp {

namespace {

constexpr int kN = 256;            // y and z lengths handled here
constexpr int kLines = 18;         // components per spectral point
constexpr int kSpecThreads = 288;  // 18 lines x 16 butterflies
constexpr int kPhaseItems = kN;    // items per phase and plane (z or ky values)

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Bounded wait until *ctr >= target; false if it gave up (or a failure was
// already recorded in *status).
__device__ __forceinline__ bool wait_count(const int* ctr, int target, const int* status) {
  for (int i = 0; i < (1 << 22); ++i) {
    if (ld_acquire_gpu(ctr) >= target) return true;
    if ((i & 63) == 63 && ld_acquire_gpu(status) != 0) return false;
    if (i > 64) __nanosleep(128);
  }
  return false;
}

__device__ __forceinline__ cpx<float> ldcg(const cpx<float>* p) {
  const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
  return cmake<float>(v.x, v.y);
}
__device__ __forceinline__ void stcg(cpx<float>* p, cpx<float> v) {
  __stcg(reinterpret_cast<float2*>(p), make_float2(v.x, v.y));
}

// Stage one of a 256-point column transform: thread (c, j) takes points
// j + 16 r (r < 16) of line c from `v`, forms their 16-point DFT and writes
// output r to position 16 j + r of the shared-memory column w.
template <int DIR>
__device__ __forceinline__ void stage1_to_smem(cpx<float> (&v)[16], cpx<float>* w, int c, int j) {
  dft16<float, DIR>(v);
#pragma unroll
  for (int r = 0; r < 16; ++r) w[(16 * j + r) * kLines + c] = v[r];
}

// Stage two: thread (c, j) takes positions 16 r + j of line c from w,
// multiplies position r by W_256^(r j) (conjugated for the inverse), forms the
// 16-point DFT; output k is point j + 16 k of the transformed column.
template <int DIR>
__device__ __forceinline__ void stage2_from_smem(const cpx<float>* w, const cpx<float>* tw, int c, int j,
                                                 cpx<float> (&v)[16]) {
  v[0] = w[j * kLines + c];
#pragma unroll
  for (int r = 1; r < 16; ++r) v[r] = cmul(w[(16 * r + j) * kLines + c], twiddle<float, DIR>(tw, r * j));
  dft16<float, DIR>(v);
}

// Y item: the y transform (direction DIR) of column (z, kx).
template <int DIR>
__device__ __forceinline__ void y_item(const CellDev<float>& c, int z, int kx, cpx<float>* w, const cpx<float>* tw,
                                       int line, int j) {
  const long long stride = (long long)c.kx * kLines;
  cpx<float>* col = c.spec + ((long long)z * c.n2 * c.kx + kx) * kLines + line;
  cpx<float> v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = ldcg(col + (long long)(j + 16 * r) * stride);
  stage1_to_smem<DIR>(v, w, line, j);
  __syncthreads();
  stage2_from_smem<DIR>(w, tw, line, j, v);
#pragma unroll
  for (int k = 0; k < 16; ++k) stcg(col + (long long)(j + 16 * k) * stride, v[k]);
}

// Z item: z forward, Green operator, z inverse of column (ky, kx).
__device__ __forceinline__ void z_item(const CellDev<float>& c, int ky, int kx, cpx<float>* w, const cpx<float>* tw,
                                       int line, int j) {
  const long long stride = (long long)c.n2 * c.kx * kLines;
  cpx<float>* col = c.spec + ((long long)ky * c.kx + kx) * kLines + line;
  cpx<float> v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = ldcg(col + (long long)(j + 16 * r) * stride);
  stage1_to_smem<-1>(v, w, line, j);
  __syncthreads();
  stage2_from_smem<-1>(w, tw, line, j, v);
  __syncthreads();  // every thread has read its stage-two inputs
#pragma unroll
  for (int k = 0; k < 16; ++k) w[(j + 16 * k) * kLines + line] = v[k];
  __syncthreads();
  // Green operator at each point kz of the column (one thread per point)
  const int kz = threadIdx.x;
  if (kz < kN) {
    cpx<float>* pt = w + kz * kLines;
    const bool nyq = (ky == c.n2 / 2) || (kz == kN / 2);
    const bool zero = (kx == 0 && ky == 0 && kz == 0);
    if (nyq || zero) {
#pragma unroll
      for (int q = 0; q < kLines; ++q) pt[q] = cmake<float>(0.f, 0.f);
    } else {
      const float x1 = c.two_pi_over_L[0] * (float)kx;
      const float x2 = c.two_pi_over_L[1] * (float)(ky <= c.n2 / 2 ? ky : ky - c.n2);
      const float x3 = c.two_pi_over_L[2] * (float)(kz <= kN / 2 ? kz : kz - kN);
      green_point<float>(c.ref, x1, x2, x3, pt, (float)c.inv_nvox);
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = w[(j + 16 * r) * kLines + line];
  __syncthreads();  // every thread has read its stage-one inputs
  stage1_to_smem<+1>(v, w, line, j);
  __syncthreads();
  stage2_from_smem<+1>(w, tw, line, j, v);
#pragma unroll
  for (int k = 0; k < 16; ++k) stcg(col + (long long)(j + 16 * k) * stride, v[k]);
}

// ctl[0]: work-queue head; ctl[1 + p * KX + g]: finished items of phase p
// (0 = Y forward, 1 = Z) of plane g.  Zeroed before every launch.
__global__ void __launch_bounds__(kSpecThreads, 2) k_spectral(CellDev<float> c, int* ctl) {
  __shared__ __align__(16) cpx<float> w[kN * kLines];
  __shared__ cpx<float> twy[kN], twz[kN];
  __shared__ int item_s;
  const int line = threadIdx.x % kLines, j = threadIdx.x / kLines;
  for (int k = threadIdx.x; k < kN; k += blockDim.x) {
    twy[k] = c.py.tw[k];
    twz[k] = c.pz.tw[k];
  }
  const int KX = c.kx;
  const long long steps = (long long)KX + 2;      // super-steps of the queue
  const long long per_step = 3ll * kPhaseItems;   // Y forward, Z, Y inverse item slots
  const long long total = steps * per_step;
  int* status = c.status;
  for (;;) {
    if (threadIdx.x == 0) item_s = atomicAdd(&ctl[0], 1);
    __syncthreads();
    const long long it = item_s;
    if (it >= total) break;
    const int t = (int)(it / per_step);
    const int rem = (int)(it - (long long)t * per_step);
    const int phase = rem / kPhaseItems;  // 0: Y forward of plane t, 1: Z of t - 1, 2: Y inverse of t - 2
    const int idx = rem - phase * kPhaseItems;
    const int g = t - phase;
    if (g < 0 || g >= KX) {
      __syncthreads();
      continue;
    }
    bool ok = true;
    if (phase > 0 && threadIdx.x == 0) {
      ok = wait_count(&ctl[1 + (phase - 1) * KX + g], kPhaseItems, status);
      if (!ok) atomicOr(status, 1);
      __threadfence();
    }
    ok = __syncthreads_and(ok) != 0;
    if (ok) {
      if (phase == 0) y_item<-1>(c, idx, g, w, twy, line, j);
      else if (phase == 1) z_item(c, idx, g, w, twz, line, j);
      else y_item<+1>(c, idx, g, w, twy, line, j);
    }
    __syncthreads();  // the item's stores are done and w may be reused
    if (phase < 2 && threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&ctl[1 + phase * KX + g], 1);
    }
  }
}

}  // namespace

size_t spectral_ctl_ints(int kx) { return 1 + 2 * (size_t)kx; }

bool spectral_fused_ok(const CellDev<float>& c) {
  return c.n1 >= 2 && c.n2 == kN && c.n3 == kN && c.kx == c.n1 / 2;
}

cudaError_t launch_spectral(const CellDev<float>& c, int* ctl, int nsm, cudaStream_t st) {
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spectral, kSpecThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
  }
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(int) * spectral_ctl_ints(c.kx), st);
  if (e != cudaSuccess) return e;
  k_spectral<<<per_sm * nsm, kSpecThreads, 0, st>>>(c, ctl);
  return cudaGetLastError();
}

}  // namespace mp
