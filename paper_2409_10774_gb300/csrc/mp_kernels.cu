// Kernels of one fixed-point iteration of the micropolar FFT scheme (sm_103a)
// and their launchers.  Spectral buffer layout: complex spec[(kz N2 + ky) KX
// + kx][18], 18 = (tau or e^: 9 comps, mu or gamma^: 9 comps), KX = N1 / 2
// (the Nyquist column kx = N1 / 2 is never stored: the Green operator zeroes
// it) or 1 when N1 == 1.
//
// One iteration (Algorithm 2 while-loop) runs
//   y-forward  ->  z-forward + Green + z-inverse  ->  y-inverse  ->  pass A
// where pass A does, row by row along x: inverse x transform, + (E, Gamma),
// Algorithm 1, error partials against the previous iterate, polarizations
// tau = t - A0 e, mu = m - B0 gamma, forward x transform.
#include "mp_kernels.cuh"

#include "mp_constitutive.cuh"
#include "mp_fft.cuh"
#include "mp_green.cuh"
#include "mp_tma.cuh"

namespace mp {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ float shfl_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double shfl_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <class T>
__device__ __forceinline__ T shfl_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class R>
__device__ __forceinline__ R signed_freq_scale(int k, int n, R two_pi_over_L) {
  const int s = (k <= n / 2) ? k : k - n;
  return two_pi_over_L * (R)s;
}

// 8 warps per block.  Registers are split between the SM's four sub-partitions
// (16 K each), so with 2 blocks per SM (4 warps per sub-partition) a thread
// may use up to 128 registers; a 9-warp block would cap it at 96.
constexpr int kThreads = 256;
// The y / z column passes: 18 components x 16 butterflies per round (a radix-16
// stage of a 256-point line is exactly one round); their registers stay low.
constexpr int kThreadsYZ = 288;
// Shared memory per block on sm_103a (opt-in maximum) and the part of it the
// dynamic tiles may use: the multi-cell kernels also hold a cell descriptor
// and a few reduction words in static shared memory.
constexpr size_t kSmemOptin = 227 * 1024;
constexpr size_t kSmemStaticReserve = 2048;
constexpr size_t kSmemBudget = kSmemOptin - kSmemStaticReserve;

// Cooperative copy of a y / z tile of CPT columns (those below ncols; col0 is
// the first), n points each, 18 complex values per (point, column): the values
// of point p of tile column j sit at g + cofs[j] + p * stride (complex units)
// and in the tile at ((p CPT + j) 18).  Loads are asynchronous 16-byte copies
// (cp.async), so every thread keeps all of its loads in flight; the caller's
// barrier follows cp_async_wait_all.
template <class R, bool TO_SMEM, int CPT>
__device__ __forceinline__ void copy_tile(cpx<R>* tile, cpx<R>* g, int n, long long col0, long long ncols,
                                          long long stride, const long long* cofs) {
  constexpr int W = 18 * (int)sizeof(cpx<R>) / 16;  // float4 per chunk
  float4* t4 = reinterpret_cast<float4*>(tile);
  const int total = n * CPT * W;
  const int nj = (int)(ncols - col0 < CPT ? ncols - col0 : CPT);
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int row = i / W, w = i - row * W;
    const int p = row / CPT, j = row - p * CPT;
    if (j >= nj) continue;
    float4* g4 = reinterpret_cast<float4*>(g + cofs[j] + p * stride) + w;
    if (TO_SMEM) cp_async16(t4 + i, g4);
    else *g4 = t4[i];
  }
  if (TO_SMEM) cp_async_wait_all();
}

// ------------------------------------------------------------------ multi-cell plumbing
// Entry owning global item g: the last e with pre[e] <= g (binary search).
__device__ __forceinline__ int find_entry(const long long* pre, int n, long long g) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Cooperative copy of a cell descriptor into shared memory (callers fence with
// barriers on both sides).
template <class R>
__device__ __forceinline__ void load_cell(CellDev<R>& dst, const CellDev<R>* src) {
  static_assert(sizeof(CellDev<R>) % 4 == 0, "descriptor size");
  const int* s4 = reinterpret_cast<const int*>(src);
  int* d4 = reinterpret_cast<int*>(&dst);
  for (int i = threadIdx.x; i < (int)(sizeof(CellDev<R>) / 4); i += blockDim.x) d4[i] = s4[i];
}

// Runs `body(cell, local_item)` over a launch's items: the single cell `c0`
// (items 0..n0-1), or, for MULTI, every entry of `w` with its cell staged in
// shared memory `cs` (reloaded when a block moves to the next cell).  A cell
// whose round control says stop (a later round of a batched window after
// its loop ended) has its items skipped; the flag only changes between
// launches, so every thread of the block reads the same value.
template <class R, bool MULTI, class Body>
__device__ __forceinline__ void for_items(const CellDev<R>& c0, long long n0, const Work<R>& w,
                                          CellDev<R>& cs, Body body) {
  if constexpr (!MULTI) {
    for (long long g = blockIdx.x; g < n0; g += gridDim.x) body(c0, g);
  } else {
    // contiguous ranges: a block's consecutive items mostly share a cell
    const long long total = w.pre[w.n_act];
    const long long per = (total + gridDim.x - 1) / gridDim.x;
    const long long g0 = (long long)blockIdx.x * per;
    const long long g1 = (g0 + per < total) ? g0 + per : total;
    if (g0 >= g1) return;
    int e = find_entry(w.pre, w.n_act, g0);
    int cur = -1;
    bool halted = false;
    for (long long g = g0; g < g1; ++g) {
      while (g >= w.pre[e + 1]) ++e;
      const int slot = w.act[e];
      if (slot != cur) {
        __syncthreads();
        load_cell(cs, w.cells + slot);
        __syncthreads();
        cur = slot;
        halted = cs.rctl != nullptr && __ldcg(&cs.rctl->stop) != 0;
      }
      if (!halted) body(cs, g - w.pre[e]);
    }
  }
}

// ------------------------------------------------------------------ y pass
// Shared memory of a y / z tile: two tiles of 18 cols_per_tile(n) lines of n
// points, the axis' twiddle table (n entries) and the tile's column offsets.
template <class R>
size_t smem_line_pass(int n) {
  return (2ull * 18 * cols_per_tile(n) + 1) * (size_t)n * sizeof(cpx<R>) + 16 * sizeof(long long);
}

// One tile = CPT consecutive columns (kz, kx), column index kz KX + kx, each
// 18 lines of length N2.  NF > 0: N2 = NF with its compile-time plan and
// CPT = cols_per_tile(NF); NF < 0: any length through the run-time plan, one
// column per tile.
template <class R, int DIR, int NF>
__device__ __forceinline__ void fft_y_tile(const CellDev<R>& c, long long tile, unsigned char* smem) {
  constexpr int CPT = NF > 0 ? cols_per_tile(NF) : 1;
  cpx<R>* b0 = reinterpret_cast<cpx<R>*>(smem);
  const int N = c.n2;
  cpx<R>* b1 = b0 + 18 * CPT * N;
  cpx<R>* tws = b1 + 18 * CPT * N;  // the axis' twiddle table, read from shared memory
  long long* cofs = reinterpret_cast<long long*>(tws + N);
  const int KX = c.kx;
  const long long stride = (long long)KX * 18;
  const long long ncols = (long long)c.n3 * KX, col0 = tile * CPT;
  if (threadIdx.x < CPT) {
    const long long col = col0 + threadIdx.x, kz = col / KX;
    cofs[threadIdx.x] = (kz * N * KX + (col - kz * KX)) * 18;
  }
  for (int k = threadIdx.x; k < N; k += blockDim.x) tws[k] = c.py.tw[k];
  __syncthreads();
  copy_tile<R, true, CPT>(b0, c.spec, N, col0, ncols, stride, cofs);
  __syncthreads();
  cpx<R>* r = tile_fft_yz<R, DIR, NF>(b0, b1, c.py, tws);
  copy_tile<R, false, CPT>(r, c.spec, N, col0, ncols, stride, cofs);
  __syncthreads();
}

// Per-tile dispatch of the run-time-length kernels on the compile-time plans.
template <class R, int DIR>
__device__ __forceinline__ void fft_y_tile_any(const CellDev<R>& c, long long tile, unsigned char* smem) {
  switch (c.n2) {
    case 256: fft_y_tile<R, DIR, 256>(c, tile, smem); break;
    case 128: fft_y_tile<R, DIR, 128>(c, tile, smem); break;
    case 64: fft_y_tile<R, DIR, 64>(c, tile, smem); break;
    case 48: fft_y_tile<R, DIR, 48>(c, tile, smem); break;
    case 32: fft_y_tile<R, DIR, 32>(c, tile, smem); break;
    case 24: fft_y_tile<R, DIR, 24>(c, tile, smem); break;
    case 16: fft_y_tile<R, DIR, 16>(c, tile, smem); break;
    default: fft_y_tile<R, DIR, -1>(c, tile, smem); break;
  }
}

// NF > 0: compiled for one column length (its transform plan unrolled);
// NF = 0: any length, dispatched per tile (multi-cell launches; every plan is
// compiled into the one kernel, so it is given the registers of two blocks
// per SM rather than spilling at three).
template <class R, int DIR, bool MULTI, int NF>
__global__ void __launch_bounds__(kThreadsYZ, NF > 0 ? 3 : 2) k_fft_y(CellDev<R> c0, Work<R> w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ CellDev<R> cs;
  for_items<R, MULTI>(c0, tiles_y(c0), w, cs, [&](const CellDev<R>& c, long long t) {
    if constexpr (NF > 0) fft_y_tile<R, DIR, NF>(c, t, smem_raw);
    else fft_y_tile_any<R, DIR>(c, t, smem_raw);
  });
}

// ------------------------------------------------------------------ z pass + Green
// One tile = CPT consecutive columns (ky, kx), column index ky KX + kx, each
// 18 lines of length N3 (NF as for the y pass).
template <class R, int NF>
__device__ __forceinline__ void green_z_tile(const CellDev<R>& c, long long tile, unsigned char* smem) {
  constexpr int CPT = NF > 0 ? cols_per_tile(NF) : 1;
  cpx<R>* b0 = reinterpret_cast<cpx<R>*>(smem);
  const int N = c.n3;
  cpx<R>* b1 = b0 + 18 * CPT * N;
  cpx<R>* tws = b1 + 18 * CPT * N;  // the axis' twiddle table, read from shared memory
  long long* cofs = reinterpret_cast<long long*>(tws + N);
  const int KX = c.kx;
  const long long stride = (long long)c.n2 * KX * 18;
  const long long ncols = (long long)c.n2 * KX, col0 = tile * CPT;
  const R scale = (R)c.inv_nvox;
  if (threadIdx.x < CPT) cofs[threadIdx.x] = (col0 + threadIdx.x) * 18;
  for (int k = threadIdx.x; k < N; k += blockDim.x) tws[k] = c.pz.tw[k];
  __syncthreads();
  copy_tile<R, true, CPT>(b0, c.spec, N, col0, ncols, stride, cofs);
  __syncthreads();
  cpx<R>* r = tile_fft_yz<R, -1, NF>(b0, b1, c.pz, tws);
  const bool even_y = (c.n2 % 2 == 0);
  const int ky0 = (int)(col0 / KX), kx0 = (int)(col0 - (long long)ky0 * KX);
  const int nj = (int)(ncols - col0 < CPT ? ncols - col0 : CPT);
  for (int i = threadIdx.x; i < N * CPT; i += blockDim.x) {
    const int kz = i / CPT, j = i - kz * CPT;
    if (j >= nj) continue;
    // column col0 + j = (ky, kx)
    int kx = kx0 + j, ky = ky0;
    if (CPT > 1) {
      const int dy = kx / KX;
      ky += dy;
      kx -= dy * KX;
    }
    cpx<R>* pt = r + i * 18;  // the point's 18 values, updated in shared memory
    // zero fluctuation on the Nyquist planes of y and z and at k = 0
    const bool nyq = (even_y && ky == c.n2 / 2) || ((N % 2 == 0) && (kz == N / 2));
    const bool zero = (kx == 0 && ky == 0 && kz == 0);
    if (nyq || zero) {
#pragma unroll
      for (int q = 0; q < 18; ++q) pt[q] = cmake<R>(R(0), R(0));
    } else {
      const R x1 = c.n1 == 1 ? R(0) : c.two_pi_over_L[0] * (R)kx;
      const R x2 = signed_freq_scale<R>(ky, c.n2, c.two_pi_over_L[1]);
      const R x3 = signed_freq_scale<R>(kz, N, c.two_pi_over_L[2]);
      green_point<R>(c.ref, x1, x2, x3, pt, scale);
    }
  }
  __syncthreads();
  cpx<R>* other = (r == b0) ? b1 : b0;
  cpx<R>* o = tile_fft_yz<R, +1, NF>(r, other, c.pz, tws);
  copy_tile<R, false, CPT>(o, c.spec, N, col0, ncols, stride, cofs);
  __syncthreads();
}

template <class R>
__device__ __forceinline__ void green_z_tile_any(const CellDev<R>& c, long long tile, unsigned char* smem) {
  switch (c.n3) {
    case 256: green_z_tile<R, 256>(c, tile, smem); break;
    case 128: green_z_tile<R, 128>(c, tile, smem); break;
    case 64: green_z_tile<R, 64>(c, tile, smem); break;
    case 48: green_z_tile<R, 48>(c, tile, smem); break;
    case 32: green_z_tile<R, 32>(c, tile, smem); break;
    case 24: green_z_tile<R, 24>(c, tile, smem); break;
    case 16: green_z_tile<R, 16>(c, tile, smem); break;
    default: green_z_tile<R, -1>(c, tile, smem); break;
  }
}

// The register file is split over the SM's four sub-partitions: 27 warps
// (three 288-thread blocks) allow 72 registers per thread, which the FP32
// single-length forms fit without spills; the others run two blocks per SM
// (18 warps, 96 registers: a few spills cost less than one block per SM).
template <class R, bool MULTI, int NF>
__global__ void __launch_bounds__(kThreadsYZ, (sizeof(R) == 4 && NF > 0) ? 3 : 2)
    k_green_z(CellDev<R> c0, Work<R> w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ CellDev<R> cs;
  for_items<R, MULTI>(c0, tiles_z(c0), w, cs, [&](const CellDev<R>& c, long long t) {
    if constexpr (NF > 0) green_z_tile<R, NF>(c, t, smem_raw);
    else green_z_tile_any<R>(c, t, smem_raw);
  });
}

// ------------------------------------------------------------------ x pass (pass A)
// Packed real transform of a row of N1 reals through a complex transform of
// length M = N1 / 2: z[n] = x[2n] + i x[2n+1].
//   forward:  X[k] = (Z[k] + conj Z[M-k]) / 2 - (i / 2) W_N1^k (Z[k] - conj Z[M-k])
//   inverse:  Z[k] = (X[k] + conj X[M-k]) + i W_N1^-k (X[k] - conj X[M-k]),  X[M] = 0
// (X[M] is the Nyquist bin, which the Green operator sets to zero; X[0] is
// real for a real row and its imaginary part is ignored).  Tiles are AoS:
// point k of line (rr, c) at [(rr M + k) 18 + c].

__device__ __forceinline__ int div_m(int q, int M, int msh) { return msh >= 0 ? (q >> msh) : (q / M); }

template <class R>
__device__ __forceinline__ void x_inverse_pre(const cpx<R>* X, cpx<R>* Z, int rows, int M, int msh,
                                              const cpx<R>* tw) {
  const int total = rows * M * 18;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int c = idx % 18;
    const int q = idx / 18;          // rr * M + k
    const int rr = div_m(q, M, msh), k = q - rr * M;
    const cpx<R>* x = X + rr * M * 18 + c;
    cpx<R> a = x[k * 18];
    if (k == 0) a.y = R(0);
    const cpx<R> b = (k == 0) ? cmake<R>(R(0), R(0)) : cconj(x[(M - k) * 18]);
    cpx<R> w = tw[k];
    w.y = -w.y;  // W_N^-k
    Z[idx] = cadd(cadd(a, b), cmuli(cmul(w, csub(a, b))));
  }
}

// The inverse pre-step fused into the first (Ns = 1) Stockham stage: each
// butterfly forms its RADIX inputs Z[j + r M / RADIX] from X (as
// x_inverse_pre does) instead of reading them from a separate pass, which
// saves one shared-memory pass and one barrier per item.
template <class R, int RADIX, int M>
__device__ __forceinline__ void stage_first_inv_packed(const cpx<R>* __restrict__ X, cpx<R>* __restrict__ out,
                                                       int rows, const cpx<R>* __restrict__ tw) {
  constexpr int nb = M / RADIX;
  constexpr int rs = M * 18;
  const int total = rows * nb * 18;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int c = idx % 18;
    const int q = idx / 18;
    const int rr = q / nb, j = q % nb;
    const cpx<R>* x = X + rr * rs + c;
    cpx<R> v[RADIX];
#pragma unroll
    for (int r = 0; r < RADIX; ++r) {
      const int k = j + r * nb;
      cpx<R> a = x[k * 18];
      if (k == 0) a.y = R(0);
      const cpx<R> b = (k == 0) ? cmake<R>(R(0), R(0)) : cconj(x[(M - k) * 18]);
      cpx<R> w = tw[k];
      w.y = -w.y;  // W_N^-k
      v[r] = cadd(cadd(a, b), cmuli(cmul(w, csub(a, b))));
    }
    if constexpr (RADIX == 3) dft3<R, +1>(v);
    else if constexpr (RADIX == 4) dft4<R, +1>(v);
    else if constexpr (RADIX == 8) dft8<R, +1>(v);
    else dft16<R, +1>(v);
    cpx<R>* dst = out + rr * rs + c + (j * RADIX) * 18;
#pragma unroll
    for (int r = 0; r < RADIX; ++r) dst[r * 18] = v[r];
  }
}

// Inverse x transform of packed rows: the spectral rows X in b0 -> the
// packed real rows (returned: b0 or b1).  Ends with a barrier.
template <class R>
__device__ cpx<R>* tile_fft_x_inv_packed(cpx<R>* b0, cpx<R>* b1, int rows, const AxisPlan<R>& p, int msh,
                                         const cpx<R>* tw) {
  auto sync_swap = [&]() {
    __syncthreads();
    cpx<R>* t = b0;
    b0 = b1;
    b1 = t;
  };
  switch (p.m) {
    case 256:
      stage_first_inv_packed<R, 8, 256>(b0, b1, rows, tw); sync_swap();
      stage_fixed<R, +1, 8, 8, 256, 2>(b0, b1, rows, tw); sync_swap();
      stage_fixed<R, +1, 4, 64, 256, 2>(b0, b1, rows, tw); sync_swap();
      return b0;
    case 128:  // as the forward transform: 16 x 8 in FP32, 8 x 4 x 4 in FP64
      if constexpr (sizeof(R) == 4) {
        stage_first_inv_packed<R, 16, 128>(b0, b1, rows, tw); sync_swap();
        stage_fixed<R, +1, 8, 16, 128, 2>(b0, b1, rows, tw); sync_swap();
      } else {
        stage_first_inv_packed<R, 8, 128>(b0, b1, rows, tw); sync_swap();
        stage_fixed<R, +1, 4, 8, 128, 2>(b0, b1, rows, tw); sync_swap();
        stage_fixed<R, +1, 4, 32, 128, 2>(b0, b1, rows, tw); sync_swap();
      }
      return b0;
    case 64:
      stage_first_inv_packed<R, 8, 64>(b0, b1, rows, tw); sync_swap();
      stage_fixed<R, +1, 8, 8, 64, 2>(b0, b1, rows, tw); sync_swap();
      return b0;
    case 32:
      stage_first_inv_packed<R, 8, 32>(b0, b1, rows, tw); sync_swap();
      stage_fixed<R, +1, 4, 8, 32, 2>(b0, b1, rows, tw); sync_swap();
      return b0;
    case 16:
      stage_first_inv_packed<R, 4, 16>(b0, b1, rows, tw); sync_swap();
      stage_fixed<R, +1, 4, 4, 16, 2>(b0, b1, rows, tw); sync_swap();
      return b0;
    case 24:
      stage_first_inv_packed<R, 8, 24>(b0, b1, rows, tw); sync_swap();
      stage_fixed<R, +1, 3, 8, 24, 2>(b0, b1, rows, tw); sync_swap();
      return b0;
    case 12:
      stage_first_inv_packed<R, 4, 12>(b0, b1, rows, tw); sync_swap();
      stage_fixed<R, +1, 3, 4, 12, 2>(b0, b1, rows, tw); sync_swap();
      return b0;
    case 8:
      stage_first_inv_packed<R, 8, 8>(b0, b1, rows, tw); sync_swap();
      return b0;
    default:
      x_inverse_pre<R>(b0, b1, rows, p.m, msh, tw);
      __syncthreads();
      return tile_fft<R, +1, 8>(b1, b0, rows, p, tw);
  }
}

template <class R>
__device__ __forceinline__ void x_forward_post(const cpx<R>* Z, cpx<R>* X, int rows, int M, int msh,
                                               const cpx<R>* tw) {
  const int total = rows * M * 18;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int c = idx % 18;
    const int q = idx / 18;
    const int rr = div_m(q, M, msh), k = q - rr * M;
    const cpx<R>* z = Z + rr * M * 18 + c;
    cpx<R> a = z[k * 18];
    cpx<R> b = cconj(z[(k == 0 ? 0 : M - k) * 18]);
    cpx<R> s = cadd(a, b), d = csub(a, b);
    cpx<R> wd = cmul(tw[k], d);
    // (s - i wd) / 2
    X[idx] = cmake<R>(R(0.5) * (s.x + wd.y), R(0.5) * (s.y - wd.x));
  }
}

// The last forward Stockham stage of a length-M transform (radix RADIX,
// Ns = M / RADIX, twiddle stride 2) fused with the packed-real post-step.
// Output k = j + Ns r of butterfly j pairs with output M - k, which butterfly
// Ns - j produces at r' = RADIX - 1 - r (butterfly 0: r' = RADIX - r mod
// RADIX; butterfly Ns / 2 pairs with itself): one thread takes butterflies j
// and Ns - j of a line, so both partners are in its registers and X goes
// straight to shared memory, without a separate post pass.
template <class R, int M, int RADIX>
__device__ __forceinline__ void x_forward_last_post(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ X,
                                                    int rows, const cpx<R>* __restrict__ tw) {
  constexpr int NS = M / RADIX, UNITS = NS / 2 + 1, LN = 18, RS = M * LN;
  const int total = rows * UNITS * LN;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int c = idx % LN;
    const int q = idx / LN;
    const int rr = q / UNITS, u = q - rr * UNITS;
    const cpx<R>* src = in + rr * RS + c;
    cpx<R>* dst = X + rr * RS + c;
    // butterfly j of the stage (as stage_fixed<R, -1, RADIX, NS, M, 2>)
    auto butterfly = [&](int j, cpx<R>(&v)[RADIX]) {
      v[0] = src[j * LN];
#pragma unroll
      for (int r = 1; r < RADIX; ++r) v[r] = cmul(src[(j + r * NS) * LN], twiddle<R, -1>(tw, 2 * r * j));
      if constexpr (RADIX == 4) dft4<R, -1>(v);
      else dft8<R, -1>(v);
    };
    // X[k] = (s - i W_N1^k d) / 2, s = Z[k] + conj(Z[M - k]), d = Z[k] - conj(Z[M - k])
    auto post = [&](int k, cpx<R> a, cpx<R> zp) {
      const cpx<R> b = cconj(zp);
      const cpx<R> sm = cadd(a, b), df = csub(a, b);
      const cpx<R> wd = cmul(tw[k], df);
      dst[k * LN] = cmake<R>(R(0.5) * (sm.x + wd.y), R(0.5) * (sm.y - wd.x));
    };
    cpx<R> v[RADIX];
    butterfly(u, v);
    if (u == 0) {
#pragma unroll
      for (int r = 0; r < RADIX; ++r) post(NS * r, v[r], v[(RADIX - r) % RADIX]);
    } else if (u == NS / 2) {
#pragma unroll
      for (int r = 0; r < RADIX; ++r) post(NS / 2 + NS * r, v[r], v[RADIX - 1 - r]);
    } else {
      cpx<R> w[RADIX];
      butterfly(NS - u, w);
#pragma unroll
      for (int r = 0; r < RADIX; ++r) {
        post(u + NS * r, v[r], w[RADIX - 1 - r]);
        post(NS - u + NS * r, w[r], v[RADIX - 1 - r]);
      }
    }
  }
}

enum PassMode { kIter = 0, kStart = 1, kXFwd = 2, kXInv = 3 };

// Shared-memory plan of pass A: a fixed header (barriers, reduction scratch,
// the block's error totals) then the buffers for `rows` rows of N1 voxels.
template <class R>
struct PassASmem {
  static constexpr size_t bar_off = 0;                                 // 2 mbarriers
  static constexpr size_t red_off = 64;                                // [16 warps][8] doubles
  static constexpr size_t acc_off = red_off + 16 * 8 * sizeof(double);  // [kErrPartials]
  static constexpr size_t head = ((acc_off + kErrPartials * sizeof(double)) + 127) / 128 * 128;
  size_t fft_bytes, b0_off, b1_off, prev_off, hist_off, pq_off, dc_off, tw_off, carry_off, total;
  __host__ __device__ PassASmem(int n1, int rows) {
    const int M = (n1 > 1) ? n1 / 2 : 1;
    const size_t nvi = (size_t)rows * n1;
    fft_bytes = (size_t)rows * M * 18 * sizeof(cpx<R>);  // multiple of 16
    b0_off = head;
    b1_off = b0_off + fft_bytes;
    prev_off = b1_off + fft_bytes;
    hist_off = prev_off + nvi * 20 * sizeof(R);
    pq_off = hist_off + nvi * 20 * sizeof(R);
    dc_off = pq_off + nvi * 2 * sizeof(double);
    tw_off = dc_off + ((18 * (size_t)rows * sizeof(R) + 15) / 16) * 16;  // x twiddles W_N1^k, k < N1
    carry_off = tw_off + ((n1 * sizeof(cpx<R>) + 15) / 16) * 16;
    // per-thread running error maxima [4][kThreads] (R), sums [4][kThreads] and
    // row sums [kThreads] (double), kept here rather than in registers
    total = carry_off + (size_t)kThreads * (4 * sizeof(R) + 5 * sizeof(double));
  }
};

// A voxel's 20-value record (previous iterate or history) between shared
// memory and registers in 16-byte pieces: records are 80 (FP32) / 160 (FP64)
// bytes apart, so per-value accesses by consecutive threads would hit the
// same banks four (two) ways; 16-byte accesses of 8 threads cover all 32 banks.
__device__ __forceinline__ void load_rec(const float* p, float* r) {
  const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float4 a = q[k];
    r[4 * k] = a.x;
    r[4 * k + 1] = a.y;
    r[4 * k + 2] = a.z;
    r[4 * k + 3] = a.w;
  }
}
__device__ __forceinline__ void load_rec(const double* p, double* r) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    const double2 a = q[k];
    r[2 * k] = a.x;
    r[2 * k + 1] = a.y;
  }
}
__device__ __forceinline__ void store_rec(float* p, const float* r) {
  float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
  for (int k = 0; k < 5; ++k) q[k] = make_float4(r[4 * k], r[4 * k + 1], r[4 * k + 2], r[4 * k + 3]);
}
__device__ __forceinline__ void store_rec(double* p, const double* r) {
  double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
  for (int k = 0; k < 10; ++k) q[k] = make_double2(r[2 * k], r[2 * k + 1]);
}

// 18-value records (the predictor base elast) are 72 / 144 bytes apart: 8- /
// 16-byte pieces.
__device__ __forceinline__ void load_rec18(const float* p, float* r) {
  const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float2 a = q[k];
    r[2 * k] = a.x;
    r[2 * k + 1] = a.y;
  }
}
__device__ __forceinline__ void load_rec18(const double* p, double* r) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double2 a = q[k];
    r[2 * k] = a.x;
    r[2 * k + 1] = a.y;
  }
}
__device__ __forceinline__ void store_rec18(float* p, const float* r) {
  float2* q = reinterpret_cast<float2*>(p);
#pragma unroll
  for (int k = 0; k < 9; ++k) q[k] = make_float2(r[2 * k], r[2 * k + 1]);
}
__device__ __forceinline__ void store_rec18(double* p, const double* r) {
  double2* q = reinterpret_cast<double2*>(p);
#pragma unroll
  for (int k = 0; k < 9; ++k) q[k] = make_double2(r[2 * k], r[2 * k + 1]);
}

// Record a timeout and leave: the caller has seen a bounded wait fail.
__device__ __forceinline__ void flag_timeout(int* status) {
  if (threadIdx.x == 0 && status) atomicOr(status, 1);
}

// One pass-A work item: `rows` consecutive rows (y, z) of a cell = a
// contiguous range of voxels and of spectral rows.  Rows, previous iterate,
// history and plastic strains move between global and shared memory by bulk
// asynchronous copies (TMA); the spectral rows are requested first so that the
// inverse transform runs while the per-voxel records are still in flight.
// Leaves the item's 8 error maxima / sums in red[0..7] (thread 0..7 views, see
// below) and its 36 row sums in `itm` (kIter only).  Returns false when a
// bounded wait expired (uniform across the block).
template <class R, int MODE, bool MULTI>
__device__ __forceinline__ bool pass_a_item(const CellDev<R>& c, long long item, unsigned char* smem_raw,
                                            uint32_t& parity, double* itm, R* tms, const R* fin_tau,
                                            const R* fin_mu, R* fout_e, R* fout_g, bool reload) {
  const int rows = c.rows_a;
  const int N1 = c.n1;
  const int M = c.kx;                 // complex entries per row (N1 / 2, or 1)
  const int msh = (M & (M - 1)) == 0 ? __ffs(M) - 1 : -1;
  const bool packed = (N1 > 1);
  const PassASmem<R> L(N1, rows);
  cpx<R>* b0 = reinterpret_cast<cpx<R>*>(smem_raw + L.b0_off);
  cpx<R>* b1 = reinterpret_cast<cpx<R>*>(smem_raw + L.b1_off);
  R* prev_s = reinterpret_cast<R*>(smem_raw + L.prev_off);
  R* hist_s = reinterpret_cast<R*>(smem_raw + L.hist_off);
  double2* pq_s = reinterpret_cast<double2*>(smem_raw + L.pq_off);
  double* red = reinterpret_cast<double*>(smem_raw + PassASmem<R>::red_off);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + PassASmem<R>::bar_off);
  R* dcin = reinterpret_cast<R*>(smem_raw + L.dc_off);
  cpx<R>* tws = reinterpret_cast<cpx<R>*>(smem_raw + L.tw_off);
  const long long nrows = (long long)c.n2 * c.n3;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool use_vox = (MODE == kIter || MODE == kStart);
  const bool use_spec_in = (MODE == kIter || MODE == kXInv);

  const long long row0 = item * rows;
  const int nr = (int)min((long long)rows, nrows - row0);
  const int nvi = nr * N1;
  const long long v0 = row0 * N1;
  // ---------------------------------------------------------- issue loads
  // the cell's constants and x twiddle table (read many times per item, from
  // shared memory): staged for the block's first item of each cell
  if (reload) {
    if (use_vox && threadIdx.x < 18) tms[threadIdx.x] = (R)c.tmean[threadIdx.x];
    for (int k = threadIdx.x; k < N1; k += blockDim.x) tws[k] = c.px.tw[k];
  }
  if (threadIdx.x == 0) {
    // the block's next item (single cell), fetched into L2 while this one runs
    if (!MULTI && item + gridDim.x < c.items_a) {
      const long long r1 = (item + gridDim.x) * rows;
      const int n1r = (int)min((long long)rows, nrows - r1);
      if (use_spec_in) bulk_prefetch_l2(c.spec + r1 * M * 18, (uint32_t)(n1r * M * 18 * sizeof(cpx<R>)));
      if (use_vox) {
        const uint32_t bp = (uint32_t)(n1r * N1 * 20 * sizeof(R));
        bulk_prefetch_l2(c.prev + r1 * N1 * 20, bp);
        bulk_prefetch_l2(c.hist + r1 * N1 * 20, bp);
        bulk_prefetch_l2(c.pq + r1 * N1 * 2, (uint32_t)(n1r * N1 * 2 * sizeof(double)));
      }
    }
    bulk_wait_read();     // the previous item's stores have read shared memory
    fence_proxy_async();  // and every thread's reads of it precede the new loads
    if (use_spec_in) {
      const uint32_t bytes = (uint32_t)(nr * M * 18 * sizeof(cpx<R>));
      mbar_arrive_expect_tx(&bars[0], bytes);
      bulk_load(b0, c.spec + row0 * M * 18, bytes, &bars[0]);
    }
    if (use_vox) {
      const uint32_t bp = (uint32_t)(nvi * 20 * sizeof(R));
      const uint32_t bq = (uint32_t)(nvi * 2 * sizeof(double));
      mbar_arrive_expect_tx(&bars[1], 2 * bp + bq);
      bulk_load(prev_s, c.prev + v0 * 20, bp, &bars[1]);
      bulk_load(hist_s, c.hist + v0 * 20, bp, &bars[1]);
      bulk_load(pq_s, c.pq + v0 * 2, bq, &bars[1]);
    }
  }
  cpx<R>* zbuf = b0;  // buffer holding the packed real rows
  // Without loads to wait for (forward-only mode), the barrier that orders
  // thread 0's wait for the previous item's bulk stores (which may still be
  // reading b0) before every thread's writes to b0 must be explicit.
  if (!use_spec_in && !use_vox) __syncthreads();
  // ---------------------------------------------------------- inverse x
  if (use_spec_in) {
    const bool ok = mbar_wait(&bars[0], parity);
    if (__syncthreads_or(!ok)) return false;
    if (MODE == kIter)
      for (int l = threadIdx.x; l < 18 * nr; l += blockDim.x) {
        const int rr = l / 18, cc = l - rr * 18;
        dcin[cc * rows + rr] = b0[rr * M * 18 + cc].x;
      }
    if (packed) {
      zbuf = tile_fft_x_inv_packed<R>(b0, b1, nr, c.px, msh, tws);
    }
  }
  if (use_vox) {
    const bool ok = mbar_wait(&bars[1], parity);
    if (__syncthreads_or(!ok)) return false;
  }
    // ---------------------------------------------------------- per voxel
    R dmax[4] = {R(0), R(0), R(0), R(0)};
    R dsum[4] = {R(0), R(0), R(0), R(0)};
    for (int lv = threadIdx.x; lv < nvi; lv += blockDim.x) {
      const int rr = lv / N1, x = lv - rr * N1;
      const int zb = (rr * M + (packed ? (x >> 1) : 0)) * 18;  // first comp of the voxel's complex
      const long long v = v0 + lv;
      // value q of the inverse-transformed row at this voxel (read where it is
      // used, so that only one level's values are in registers at a time)
      const R* zv = reinterpret_cast<const R*>(zbuf + zb) + ((packed && (x & 1)) ? 1 : 0);
      if (MODE == kXInv) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          fout_e[v * 9 + q] = zv[2 * q];
          fout_g[v * 9 + q] = zv[2 * (9 + q)];
        }
        continue;
      }
      // value q of this voxel goes to the real (even x) or imaginary (odd x)
      // part of its packed complex entry
      R* zr = reinterpret_cast<R*>(zbuf + zb) + ((packed && (x & 1)) ? 1 : 0);
      if (!packed) {
#pragma unroll
        for (int q = 0; q < 18; ++q) zr[2 * q + 1] = R(0);
      }
      if (MODE == kXFwd) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
          zr[2 * q] = fin_tau[v * 9 + q];
          zr[2 * (9 + q)] = fin_mu[v * 9 + q];
        }
        continue;
      }
      // The voxel's two levels (Algorithm 1's macro level: e, t, f_t; micro
      // level: gamma, m, f_m) are independent: they run one after the other so
      // that only one level's tensors are held in registers at a time.  Records
      // (80 bytes apart) move in 16-byte pieces:
      //   previous iterate  {e0-3} {e4-7} {e8 g0 g1 g2} {g3-6} {g7 g8 f_t f_m}
      //   history           {ht0-3} {ht4-7} {ht8 hm0 hm1 hm2} {hm3-6} {hm7 hm8 phase 0}
      float4* pv4 = reinterpret_cast<float4*>(prev_s + lv * 20);
      const float4* hv4 = reinterpret_cast<const float4*>(hist_s + lv * 20);
      R* pv = prev_s + lv * 20;
      const R* hv = hist_s + lv * 20;
      const PhaseDev<R>& P = c.phases[(int)hv[18]];
      const double2 pq = pq_s[lv];
      const R fto = pv[18], fmo = pv[19];
      const R a0 = c.ref.mu + c.ref.kap, b0 = c.ref.mu - c.ref.kap;
      const bool din = MODE == kIter && c.delta_in != 0, dout = MODE == kIter && c.delta_out != 0;
      const R* sv = c.src ? c.src + v * 18 : nullptr;
      R ft, fm, e8;
      // ---- macro level
      {
        R e[9], eo[9], ht[9], t[9];
        if constexpr (sizeof(R) == 4) {
          const float4 q0 = pv4[0], q1 = pv4[1], q2 = pv4[2];
          const float4 h0 = hv4[0], h1 = hv4[1], h2 = hv4[2];
          eo[0] = q0.x; eo[1] = q0.y; eo[2] = q0.z; eo[3] = q0.w;
          eo[4] = q1.x; eo[5] = q1.y; eo[6] = q1.z; eo[7] = q1.w; eo[8] = q2.x;
          ht[0] = h0.x; ht[1] = h0.y; ht[2] = h0.z; ht[3] = h0.w;
          ht[4] = h1.x; ht[5] = h1.y; ht[6] = h1.z; ht[7] = h1.w; ht[8] = h2.x;
        } else {
#pragma unroll
          for (int q = 0; q < 9; ++q) {
            eo[q] = pv[q];
            ht[q] = hv[q];
          }
        }
        // de9: the strain change that enters the polarization, e - E (full
        // form) or e^i - e^{i-1} (increment form)
        R de9[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) de9[q] = (MODE == kIter) ? zv[2 * q] : R(0);
#pragma unroll
        for (int q = 0; q < 9; ++q) e[q] = (MODE == kIter) ? (din ? eo[q] : c.E[q]) + de9[q] : eo[q];
        double pn = pq.x;
        // the pass needs the scale factor only (p is formed at the commit)
        return_macro<R, sizeof(R) == 4 ? 1 : 2>(P, e, ht, pn, t, pn, ft);
        if (MODE == kIter) {
          if (dout) {
#pragma unroll
            for (int q = 0; q < 9; ++q) de9[q] = e[q] - eo[q];
          }
          const R trd = de9[0] + de9[4] + de9[8];
          // previous stresses rebuilt from the stored strains and scale factor
          // (t = tr/3 d + f_t dev(t_trial)), in the same operation order
          const R tre = (eo[0] + eo[4]) + eo[8];
          const R vol = vol_of(trial_t(P, ht[0], eo[0], eo[0], true, tre), trial_t(P, ht[4], eo[4], eo[4], true, tre),
                               trial_t(P, ht[8], eo[8], eo[8], true, tre));
          R de = R(0), dt = R(0);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int l = 0; l < 3; ++l) {
              const int i = 3 * k + l, j = 3 * l + k;
              const R to = scaled_t(trial_t(P, ht[i], eo[i], eo[j], k == l, tre), k == l, vol, fto);
              const R d1 = e[i] - eo[i], d2 = t[i] - to;
              de += d1 * d1;
              dt += d2 * d2;
              // full form: tau - tau_c = (t - <t>_prev) - A0 (e - E); the
              // constants tau_c = <t>_prev - A0 E only change the k = 0 term,
              // which the Green operator drops, and the transforms then round
              // relative to a field of fluctuations.  Increment form:
              // tau(e^i) - tau(e^{i-1}) = (t - t_prev) - A0 (e^i - e^{i-1}).
              R ae = a0 * de9[i] + b0 * de9[j];
              if (k == l) ae += c.ref.lam * trd;
              // manufactured source (eq. manufactured_polarization_stress); it
              // cancels in the increment form
              if (sv && !dout) ae += sv[i];
              zr[2 * i] = (t[i] - (dout ? to : tms[i])) - ae;
            }
          }
          de = sqrt(de);
          dt = sqrt(dt);
          dmax[0] = max(dmax[0], de); dmax[1] = max(dmax[1], dt);
          dsum[0] += de; dsum[1] += dt;
        } else {
#pragma unroll
          for (int q = 0; q < 9; ++q) de9[q] = e[q] - c.E[q];
          const R trd = de9[0] + de9[4] + de9[8];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int l = 0; l < 3; ++l) {
              const int i = 3 * k + l, j = 3 * l + k;
              R ae = a0 * de9[i] + b0 * de9[j];
              if (k == l) ae += c.ref.lam * trd;
              if (sv) ae += sv[i];
              zr[2 * i] = (t[i] - tms[i]) - ae;
            }
          }
        }
        if constexpr (sizeof(R) == 4) {
          pv4[0] = make_float4(e[0], e[1], e[2], e[3]);
          pv4[1] = make_float4(e[4], e[5], e[6], e[7]);
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) pv[q] = e[q];
        }
        e8 = e[8];
      }
      // ---- micro level
      {
        R g[9], go[9], hm[9], m[9];
        if constexpr (sizeof(R) == 4) {
          const float4 q2 = pv4[2], q3 = pv4[3], q4 = pv4[4];
          const float4 h2 = hv4[2], h3 = hv4[3], h4 = hv4[4];
          go[0] = q2.y; go[1] = q2.z; go[2] = q2.w; go[3] = q3.x; go[4] = q3.y;
          go[5] = q3.z; go[6] = q3.w; go[7] = q4.x; go[8] = q4.y;
          hm[0] = h2.y; hm[1] = h2.z; hm[2] = h2.w; hm[3] = h3.x; hm[4] = h3.y;
          hm[5] = h3.z; hm[6] = h3.w; hm[7] = h4.x; hm[8] = h4.y;
        } else {
#pragma unroll
          for (int q = 0; q < 9; ++q) {
            go[q] = pv[9 + q];
            hm[q] = hv[9 + q];
          }
        }
        R dg9[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) dg9[q] = (MODE == kIter) ? zv[2 * (9 + q)] : R(0);
#pragma unroll
        for (int q = 0; q < 9; ++q) g[q] = (MODE == kIter) ? (din ? go[q] : c.G[q]) + dg9[q] : go[q];
        double qn = pq.y;
        return_micro<R, sizeof(R) == 4 ? 1 : 2>(P, g, hm, qn, m, qn, fm);
        if (MODE == kIter) {
          if (dout) {
#pragma unroll
            for (int q = 0; q < 9; ++q) dg9[q] = g[q] - go[q];
          }
          const R trd = dg9[0] + dg9[4] + dg9[8];
          const R trg = (go[0] + go[4]) + go[8];
          R dg = R(0), dm = R(0);
#pragma unroll
          for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int l = 0; l < 3; ++l) {
              const int i = 3 * k + l, j = 3 * l + k;
              const R mo = trial_m(P, hm[i], go[i], go[j], k == l, trg) * fmo;
              const R d3 = g[i] - go[i], d4 = m[i] - mo;
              dg += d3 * d3;
              dm += d4 * d4;
              R bg = c.ref.beta * dg9[i] + c.ref.gamma * dg9[j];
              if (k == l) bg += c.ref.alpha * trd;
              if (sv && !dout) bg += sv[9 + i];
              zr[2 * (9 + i)] = (m[i] - (dout ? mo : tms[9 + i])) - bg;
            }
          }
          dg = sqrt(dg);
          dm = sqrt(dm);
          dmax[2] = max(dmax[2], dg); dmax[3] = max(dmax[3], dm);
          dsum[2] += dg; dsum[3] += dm;
        } else {
#pragma unroll
          for (int q = 0; q < 9; ++q) dg9[q] = g[q] - c.G[q];
          const R trd = dg9[0] + dg9[4] + dg9[8];
#pragma unroll
          for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int l = 0; l < 3; ++l) {
              const int i = 3 * k + l, j = 3 * l + k;
              R bg = c.ref.beta * dg9[i] + c.ref.gamma * dg9[j];
              if (k == l) bg += c.ref.alpha * trd;
              if (sv) bg += sv[9 + i];
              zr[2 * (9 + i)] = (m[i] - tms[9 + i]) - bg;
            }
          }
        }
        if constexpr (sizeof(R) == 4) {
          pv4[2] = make_float4(e8, g[0], g[1], g[2]);
          pv4[3] = make_float4(g[3], g[4], g[5], g[6]);
          pv4[4] = make_float4(g[7], g[8], ft, fm);
        } else {
          pv[8] = e8;
#pragma unroll
          for (int q = 0; q < 9; ++q) pv[9 + q] = g[q];
          pv[18] = ft;
          pv[19] = fm;
        }
      }
    }
    if (MODE == kXInv) {
    __syncthreads();
    parity ^= 1u;
    return true;
  }
  // the new iterate goes back to global memory while the forward transform runs
  fence_proxy_async();
  __syncthreads();
  if (use_vox && threadIdx.x == 0) {
    bulk_store(c.prev + v0 * 20, prev_s, (uint32_t)(nvi * 20 * sizeof(R)));
    bulk_commit();
  }
  // ---------------------------------------------------------- forward x
  cpx<R>* X;
  if (sizeof(R) == 4 && packed && (M == 128 || M == 64 || M == 32)) {
    // FP32: the first stage of the compile-time plan, then its last stage
    // fused with the post-step (128: 16 x 8, 64: 8 x 8, 32: 8 x 4)
    cpx<R>* other = (zbuf == b0) ? b1 : b0;
    if (M == 128) stage_fixed<R, -1, 16, 1, 128, 2>(zbuf, other, nr, tws);
    else if (M == 64) stage_fixed<R, -1, 8, 1, 64, 2>(zbuf, other, nr, tws);
    else stage_fixed<R, -1, 8, 1, 32, 2>(zbuf, other, nr, tws);
    __syncthreads();
    if (M == 128) x_forward_last_post<R, 128, 8>(other, zbuf, nr, tws);
    else if (M == 64) x_forward_last_post<R, 64, 8>(other, zbuf, nr, tws);
    else x_forward_last_post<R, 32, 4>(other, zbuf, nr, tws);
    X = zbuf;
  } else if (packed) {
    cpx<R>* other = (zbuf == b0) ? b1 : b0;
    cpx<R>* Z = tile_fft_x<R, -1>(zbuf, other, nr, c.px, tws);
    cpx<R>* dst = (Z == b0) ? b1 : b0;
    x_forward_post<R>(Z, dst, nr, M, msh, tws);
    X = dst;
  } else {
    X = zbuf;
  }
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    bulk_store(c.spec + row0 * M * 18, X, (uint32_t)(nr * M * 18 * sizeof(cpx<R>)));
    bulk_commit();
  }
  // ---------------------------------------------------------- error partials of the item
  // Per-voxel norms of the FP32 (or FP64) field differences are formed in the
  // field type; their maxima are exact in any precision, and their sums (the
  // average measure) and the row sums behind the means are accumulated in FP64.
  if (MODE == kIter) {
    // the sums only enter the average measure (eq. err_average)
    const bool want_sum = c.err_kind != 0;
    if constexpr (MULTI) {
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const R mx = shfl_max(dmax[a]);
        const double sm = want_sum ? shfl_sum((double)dsum[a]) : 0.0;
        if (lane == 0) {
          red[warp * 8 + a] = (double)mx;
          red[warp * 8 + 4 + a] = sm;
        }
      }
    } else {
      R* cmx = reinterpret_cast<R*>(smem_raw + L.carry_off);
      double* csm = reinterpret_cast<double*>(cmx + 4 * kThreads);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        R& m = cmx[a * kThreads + threadIdx.x];
        m = max(m, dmax[a]);
        if (want_sum) csm[a * kThreads + threadIdx.x] += (double)dsum[a];
      }
    }
    // Row sums.  With the unnormalised inverse along x, sum_x e~ = N1 X_in[0],
    // so sum_x e = N1 (E + X_in[0]); the forward DC is sum_x tau.
    double rsum = 0.0;
    const int q = threadIdx.x - 32;
    if (q >= 0 && q < 36) {
      if (q < 18) {
        const double mean = (double)((q < 9) ? c.E[q] : c.G[q - 9]);
        for (int rr = 0; rr < nr; ++rr) rsum += (double)N1 * (mean + (double)dcin[q * rows + rr]);
      } else {
        for (int rr = 0; rr < nr; ++rr) rsum += (double)X[rr * M * 18 + (q - 18)].x;
      }
      if constexpr (!MULTI)
        reinterpret_cast<double*>(smem_raw + L.carry_off + kThreads * (4 * sizeof(R) + 4 * sizeof(double)))[threadIdx.x] += rsum;
    }
    if constexpr (MULTI) {
      __syncthreads();
      const int nwarp = blockDim.x >> 5;
      if (threadIdx.x < 8) {
        double a = red[threadIdx.x];
        for (int w = 1; w < nwarp; ++w) {
          const double vv = red[w * 8 + threadIdx.x];
          a = (threadIdx.x < 4) ? fmax(a, vv) : a + vv;
        }
        itm[threadIdx.x] = a;
      } else if (q >= 0 && q < 36) {
        itm[8 + q] = rsum;
      }
    }
  }
  __syncthreads();
  parity ^= 1u;
  return true;
}

// Pass A over a cell (single: per-block error totals in `partials`) or over
// the entries of a multi-cell launch (per-item partials in each cell's ipart).
template <class R, int MODE, bool MULTI>
__global__ void __launch_bounds__(kThreads, (sizeof(R) == 4 ? 2 : 1))
    k_pass_a(CellDev<R> c0, Work<R> w, double* partials, const R* fin_tau, const R* fin_mu,
             R* fout_e, R* fout_g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ CellDev<R> cs;
  __shared__ double itm[kErrPartials];
  __shared__ R tms[18];  // <t>, <m> of the cell's previous iteration (subtracted constants)
  double* acc = reinterpret_cast<double*>(smem_raw + PassASmem<R>::acc_off);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + PassASmem<R>::bar_off);
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_barrier_init();
  }
  for (int i = threadIdx.x; i < kErrPartials; i += blockDim.x) acc[i] = 0.0;
  __syncthreads();
  uint32_t parity = 0;
  bool failed = false;
  int* status = c0.status;
  // the per-thread carries (error maxima and sums, row sums of threads 32..67)
  // start at zero; they sit after the item buffers for the block's row count
  const PassASmem<R> SL(c0.n1 > 0 ? c0.n1 : 1, c0.rows_a > 0 ? c0.rows_a : 1);
  if constexpr (!MULTI) {
    R* cmx = reinterpret_cast<R*>(smem_raw + SL.carry_off);
    double* csm = reinterpret_cast<double*>(cmx + 4 * kThreads);
    for (int a = 0; a < 4; ++a) {
      cmx[a * kThreads + threadIdx.x] = R(0);
      csm[a * kThreads + threadIdx.x] = 0.0;
    }
    csm[4 * kThreads + threadIdx.x] = 0.0;
  }
  for_items<R, MULTI>(c0, c0.items_a, w, cs, [&](const CellDev<R>& c, long long item) {
    if (failed) {
      flag_timeout(c.status);  // every cell with a skipped item reports the failure
      return;
    }
    // single cell: the block's first item stages the cell's tables; several
    // cells: every item does (its cell may differ from the previous one's)
    const bool reload = MULTI || item == (long long)blockIdx.x;
    if (!pass_a_item<R, MODE, MULTI>(c, item, smem_raw, parity, itm, tms, fin_tau, fin_mu, fout_e, fout_g,
                                     reload)) {
      failed = true;
      status = c.status;
      return;
    }
    if (MODE == kIter) {
      if constexpr (MULTI) {
        for (int i = threadIdx.x; i < kErrPartials; i += blockDim.x)
          c.ipart[item * kErrPartials + i] = itm[i];
        __syncthreads();
      }
    }
  });
  if (MODE == kIter && !MULTI && !failed) {
    // the block's error maxima and sums from the per-thread carries
    double* red = reinterpret_cast<double*>(smem_raw + PassASmem<R>::red_off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const R* cmx = reinterpret_cast<const R*>(smem_raw + SL.carry_off);
      const double* csm = reinterpret_cast<const double*>(cmx + 4 * kThreads);
      const R mx = shfl_max(cmx[a * kThreads + threadIdx.x]);
      const double sm = shfl_sum(csm[a * kThreads + threadIdx.x]);
      if (lane == 0) {
        red[warp * 8 + a] = (double)mx;
        red[warp * 8 + 4 + a] = sm;
      }
    }
    __syncthreads();
    if (threadIdx.x < 8) {
      double a = red[threadIdx.x];
      for (int wi = 1; wi < (int)(blockDim.x >> 5); ++wi) {
        const double vv = red[wi * 8 + threadIdx.x];
        a = (threadIdx.x < 4) ? fmax(a, vv) : a + vv;
      }
      acc[threadIdx.x] = a;
    }
    const int q = threadIdx.x - 32;
    if (q >= 0 && q < 36)
      acc[8 + q] = reinterpret_cast<const double*>(smem_raw + SL.carry_off + kThreads * (4 * sizeof(R) + 4 * sizeof(double)))[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) bulk_wait_all();
  if (failed) {
    // wait (bounded) for this block's loads still in flight, then report
    if (threadIdx.x == 0) {
      if (MODE == kIter || MODE == kXInv) mbar_wait(&bars[0], parity);
      if (MODE == kIter || MODE == kStart) mbar_wait(&bars[1], parity);
    }
    __syncthreads();
    flag_timeout(status);
    return;
  }
  if (MODE == kIter && !MULTI) {
    for (int i = threadIdx.x; i < kErrPartials; i += blockDim.x)
      partials[(long long)blockIdx.x * kErrPartials + i] = acc[i];
  }
}

// ------------------------------------------------------------------ iteration error
// eq. err with eq. err_local (max) or eq. err_average (mean).  Denominators
// ||<a>|| are floored by their dimensional partner through the voxel size h
// (den_e >= h |<gamma>|, den_gamma >= |<e>| / h, den_t >= |<m>| / h,
// den_m >= h |<t>|), since ||<gamma>|| = 0 whenever the mean curvature is zero,
// each ||<a>|| taken as the larger of its value now and the largest of the
// converged increments so far (a cyclic load passes through zero means).
// out[0] = err, out[1..4] = err_e, err_t, err_gamma, err_m, out[5] = status.
template <class R>
__device__ void finish_err(const CellDev<R>& c, const double* s, int err_kind, double* out) {
    const double iv = c.inv_nvox;
    double me[9], mg[9], mt[9], mm[9];
    for (int q = 0; q < 9; ++q) {
      me[q] = s[8 + q] * iv;
      mg[q] = s[17 + q] * iv;
    }
    // The transformed polarization was tau - tau_c = (t - T_c) - A0 (e - E) (T_c =
    // c.tmean as read by pass A), so <t> = <tau - tau_c> + T_c + A0 (<e> - E) and
    // likewise <m>; <t>, <m> then become the constants of the next iteration.
    // In the increment form it was (t - t_prev) - A0 (e - e_prev), so the same
    // formula holds with T_c = <t_prev> (the unrounded last mean) and
    // <e_prev> = E.
    const double lam = c.ref.lam, mu = c.ref.mu, kap = c.ref.kap;
    const double al = c.ref.alpha, be = c.ref.beta, ga = c.ref.gamma;
    double xe[9], xg[9];
    for (int q = 0; q < 9; ++q) {
      xe[q] = me[q] - (double)c.E[q];
      xg[q] = mg[q] - (double)c.G[q];
    }
    const double tre = xe[0] + xe[4] + xe[8], trg = xg[0] + xg[4] + xg[8];
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) {
        const int i = 3 * k + l, j = 3 * l + k;
        const double tc = c.delta_out ? c.tmean[i] : (double)(R)c.tmean[i];
        const double mc = c.delta_out ? c.tmean[9 + i] : (double)(R)c.tmean[9 + i];
        mt[i] = s[26 + i] * iv + tc + (mu + kap) * xe[i] + (mu - kap) * xe[j] + (k == l ? lam * tre : 0.0);
        mm[i] = s[35 + i] * iv + mc + be * xg[i] + ga * xg[j] + (k == l ? al * trg : 0.0);
      }
    for (int q = 0; q < 9; ++q) {
      c.tmean[q] = mt[q];
      c.tmean[9 + q] = mm[q];
    }
    double ne = 0, ng = 0, nt = 0, nm = 0;
    for (int q = 0; q < 9; ++q) {
      ne += me[q] * me[q]; ng += mg[q] * mg[q]; nt += mt[q] * mt[q]; nm += mm[q] * mm[q];
    }
    ne = sqrt(ne); ng = sqrt(ng); nt = sqrt(nt); nm = sqrt(nm);
    // magnitudes: the means now or, if larger, the largest of the converged
    // increments so far (a cyclic load passing through a zero mean)
    ne = fmax(ne, c.tmean[18]);
    nt = fmax(nt, c.tmean[19]);
    ng = fmax(ng, c.tmean[20]);
    nm = fmax(nm, c.tmean[21]);
    const double h = c.h;
    const double den[4] = {fmax(ne, h * ng), fmax(nt, nm / h), fmax(ng, ne / h), fmax(nm, h * nt)};
    double err = 0.0;
    for (int a = 0; a < 4; ++a) {
      const double num = (err_kind == 0) ? s[a] : s[4 + a] * iv;
      double ea;
      if (den[a] == 0.0) ea = (num == 0.0) ? 0.0 : INFINITY;
      else ea = num / den[a];
      if (!(ea <= err)) err = ea;  // propagates NaN
      out[1 + a] = ea;
    }
    out[0] = err;
    out[5] = c.status ? (double)(*c.status) : 0.0;
}

// Fixed-order FP64 fold of `nparts` partial records (max for the first four
// entries, sums for the rest; the block partials of a single cell, or a
// batched cell's per-item records) by one block; the total lands in s[].
// Thread (q, g) folds value q over the g-th of kFoldGroups contiguous record
// ranges in record order (neighbouring q read neighbouring doubles), then
// thread q folds the groups in order.
constexpr int kFoldGroups = 5;  // 5 x 44 = 220 of the 256 threads
__device__ __forceinline__ void fold_items(const double* partials, long long nparts, double* s,
                                           double (*part)[kErrPartials]) {
  const int t = threadIdx.x;
  if (t < kFoldGroups * kErrPartials) {
    const int q = t % kErrPartials, g = t / kErrPartials;
    const long long per = (nparts + kFoldGroups - 1) / kFoldGroups;
    const long long b0 = (long long)g * per;
    const long long b1 = (b0 + per < nparts) ? b0 + per : nparts;
    double v = 0.0;
    for (long long b = b0; b < b1; ++b) {
      const double x = partials[b * kErrPartials + q];
      v = (q < 4) ? fmax(v, x) : v + x;
    }
    part[g][q] = v;
  }
  __syncthreads();
  if (t < kErrPartials) {
    double v = part[0][t];
    for (int g = 1; g < kFoldGroups; ++g) v = (t < 4) ? fmax(v, part[g][t]) : v + part[g][t];
    s[t] = v;
  }
  __syncthreads();
}

template <class R>
__global__ void __launch_bounds__(256) k_reduce_err(CellDev<R> c, const double* partials, int nparts,
                                                    int err_kind, double* out) {
  __shared__ double s[kErrPartials];
  __shared__ double part[kFoldGroups][kErrPartials];
  fold_items(partials, nparts, s, part);
  if (threadIdx.x == 0) finish_err<R>(c, s, err_kind, out);
}

// The same reduction, deciding the fixed-point loop on the device (Algorithm 2's
// while test) for a launch inside a conditional WHILE node: out[6] counts the
// iterations of the loop; the loop continues while no failure is recorded,
// err is finite, err <= div_limit, err > tol, fewer than max_iter iterations
// ran and (stag > 0) the stagnation watch (stall_step with window stag) has
// not tripped: out[7], out[8] hold the last low and its iteration, out[10]
// the longest gap between lows, out[9] = 1 records a stop by the watch.
template <class R>
__global__ void __launch_bounds__(256) k_reduce_err_loop(CellDev<R> c, const double* partials, int nparts,
                                                         int err_kind, double* out, double tol, int max_iter,
                                                         double div_limit, int stag, int adapt,
                                                         cudaGraphConditionalHandle handle) {
  __shared__ double s[kErrPartials];
  __shared__ double part[kFoldGroups][kErrPartials];
  fold_items(partials, nparts, s, part);
  if (threadIdx.x == 0) {
    finish_err<R>(c, s, err_kind, out);
    const int it = (int)out[6] + 1;
    out[6] = (double)it;
    const double err = out[0];
    bool go = out[5] == 0.0 && isfinite(err) && err <= div_limit && err > tol && it < max_iter;
    if (go && stag > 0) {
      double ref_err = out[7];
      int it_ref = (int)out[8], gap = (int)out[10];
      if (stall_step(err, it, stag, adapt != 0, ref_err, it_ref, gap)) {
        go = false;
        out[9] = 1.0;
      }
      out[7] = ref_err;
      out[8] = (double)it_ref;
      out[10] = (double)gap;
    }
    cudaGraphSetConditional(handle, go ? 1u : 0u);
  }
}

// One block per entry: the cell's per-item partials in item order.
// Algorithm 2's loop test for one batched cell after an iteration whose error
// row is e (err, four terms, status), with the batched engine's FP32
// stagnation watch; the same comparisons, in the same order and arithmetic,
// as the host's replay of the rows.
__device__ void round_decide(RoundCtl& rc, const double* e) {
  const double err = e[0];
  rc.it += 1;
  rc.rounds += 1;
  bool stop = false;
  if (e[5] != 0.0) {
    stop = true;  // a bounded wait expired
  } else if (!isfinite(err) || err > rc.div_limit) {
    stop = true;  // diverged
  } else {
    const bool more = rc.target >= 0 ? rc.it < rc.target : err > rc.tol;
    if (!more) {
      stop = true;  // converged, or the prescribed count reached
    } else if (rc.target < 0 && rc.it >= rc.max_iter) {
      stop = true;  // not converged
    } else if (rc.stag_iters > 0) {
      // the host switches the schedule where the watch trips
      if (stall_step(err, rc.it, rc.stag_iters, rc.adapt != 0, rc.ref_err, rc.it_ref, rc.gap)) stop = true;
    }
  }
  if (rc.rounds >= rc.max_rounds) stop = true;
  rc.stop = stop ? 1 : 0;
}

template <class R>
__global__ void __launch_bounds__(256) k_reduce_err_multi(Work<R> w) {
  __shared__ double s[kErrPartials];
  __shared__ double part[kFoldGroups][kErrPartials];
  __shared__ CellDev<R> cs;
  load_cell(cs, w.cells + w.act[blockIdx.x]);
  __syncthreads();
  RoundCtl* rc = cs.rctl;
  if (rc != nullptr && __ldcg(&rc->stop) != 0) return;  // uniform: one flag per block
  fold_items(cs.ipart, cs.items_a, s, part);
  if (threadIdx.x == 0) {
    if (rc != nullptr) {
      double* out = rc->rows + 8 * rc->rounds;
      finish_err<R>(cs, s, cs.err_kind, out);
      round_decide(*rc, out);
    } else {
      finish_err<R>(cs, s, cs.err_kind, cs.err_out);
    }
  }
}

// ------------------------------------------------------------------ state set-up
// Zero initial state (Algorithm 2 initialisation) and the first predictor
// e = E, gamma = Gamma of the first load increment.  Items: 256-voxel chunks.
template <class R>
__device__ __forceinline__ void init_chunk(const CellDev<R>& c, long long chunk) {
  const long long v = chunk * 256 + threadIdx.x;
  if (threadIdx.x >= 256 || v >= c.nvox) return;
  R* pv = c.prev + v * 20;
  R* hv = c.hist + v * 20;
  R* el = c.elast + v * 18;
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    pv[q] = c.E[q];
    pv[9 + q] = c.G[q];
  }
  pv[18] = R(1);
  pv[19] = R(1);
#pragma unroll
  for (int q = 0; q < 18; ++q) {
    hv[q] = R(0);
    el[q] = R(0);
  }
  hv[18] = (R)c.phase[v];  // phase id travels with the history record
  hv[19] = R(0);
  reinterpret_cast<double2*>(c.pq)[v] = make_double2(0.0, 0.0);
}

template <class R, bool MULTI>
__global__ void __launch_bounds__(256) k_init(CellDev<R> c0, Work<R> w) {
  __shared__ CellDev<R> cs;
  for_items<R, MULTI>(c0, (c0.nvox + 255) / 256, w, cs,
                      [&](const CellDev<R>& c, long long chunk) { init_chunk<R>(c, chunk); });
}

// ------------------------------------------------------------------ commit
// Error-free sum of two single-precision values (Knuth's TwoSum): s + err =
// a + b exactly.  Accumulating x into (hi, lo) as hi, err = TwoSum(hi, x),
// lo += err is compensated summation: the pair carries the running sum to
// about 2^-48 of its magnitude, so per-thread sums of FP32 values lose
// nothing against an FP64 accumulator at the voxel counts of one thread, at
// six single-precision additions instead of one FP64 addition.
__device__ __forceinline__ void two_sum_acc(float2& acc, float x) {
  const float s = __fadd_rn(acc.x, x);
  const float bb = __fsub_rn(s, acc.x);
  const float err = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  acc.x = s;
  acc.y = __fadd_rn(acc.y, err);
}

// Algorithm 2, end of a load increment: the converged iterate becomes the
// history of Algorithm 1; homogenized sums; when c.predict, the linear-
// extrapolation predictor of the next increment, e' = e_n + ratio (e_n - e_{n-1}).
// Per 256-voxel chunk: sums of t (9), m (9), e (9), gamma (9), p, q, t_eq, m_eq
// in that order (p and q are FP64 values, the others field-type values).
// COLS: instead of reducing the chunk, add the thread's values to its own
// column of `cols` ([kAvgPartials][blockDim] 8-byte slots; single-cell
// commit): FP64 columns for FP64 fields and for p, q, compensated FP32
// (hi, lo) pairs for the field-type values of FP32 fields.
template <class R, bool COLS>
__device__ __forceinline__ void commit_chunk(const CellDev<R>& c, long long chunk, double* out40,
                                             double (*red)[kAvgPartials], double* cols) {
  R val[kAvgPartials];  // [36], [37] unused (p, q are FP64)
#pragma unroll
  for (int i = 0; i < kAvgPartials; ++i) val[i] = R(0);
  double p = 0.0, q = 0.0;
  const long long v = chunk * 256 + threadIdx.x;
  if (threadIdx.x < 256 && v < c.nvox) {
    // records move in 16- / 8-byte pieces (they are 80 / 72 bytes apart)
    R* pv = c.prev + v * 20;
    R* hv = c.hist + v * 20;
    R pr[20], hr[20];
    load_rec(pv, pr);
    load_rec(hv, hr);
    const R* e = pr;
    const R* g = pr + 9;
    const PhaseDev<R>& P = c.phases[(int)hr[18]];
    double2 pq = reinterpret_cast<const double2*>(c.pq)[v];
    R t[9], m[9];
    R ft, fm;
    radial_return<R>(P, e, g, hr, hr + 9, pq.x, pq.y, t, m, p, q, ft, fm);
    R ae[9], bg[9];
    apply_A<R>(P.lam, P.mu, P.kap, e, ae);
    apply_B<R>(P.alpha, P.beta, P.gamma, g, bg);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      val[i] = t[i];
      val[9 + i] = m[i];
      val[18 + i] = e[i];
      val[27 + i] = g[i];
      hr[i] = t[i] - ae[i];
      hr[9 + i] = m[i] - bg[i];
    }
    store_rec(hv, hr);
    reinterpret_cast<double2*>(c.pq)[v] = make_double2(p, q);
    equivalents<R>(P, t, m, val[38], val[39]);
    if (c.predict) {
      const R ratio = (R)c.ratio;
      R* el = c.elast + v * 18;
      R old[18];
      load_rec18(el, old);
      store_rec18(el, pr);  // e, gamma (the first 18 values of the iterate record)
#pragma unroll
      for (int i = 0; i < 18; ++i) pr[i] = pr[i] + ratio * (pr[i] - old[i]);
      store_rec(pv, pr);    // the predictor, with the last scale factors
    }
  }
  const int bd = (int)blockDim.x;
  if constexpr (COLS) {
    // thread-private columns: no cross-thread work per chunk
    double* dc = cols + threadIdx.x;
#pragma unroll
    for (int i = 0; i < kAvgPartials; ++i) {
      if (i == 36) {
        dc[i * bd] += p;
      } else if (i == 37) {
        dc[i * bd] += q;
      } else if constexpr (sizeof(R) == 4) {
        float2* fc = reinterpret_cast<float2*>(dc + i * bd);
        float2 a = *fc;
        two_sum_acc(a, (float)val[i]);
        *fc = a;
      } else {
        dc[i * bd] += (double)val[i];
      }
    }
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < kAvgPartials; ++i) {
    const double x = (i == 36) ? p : (i == 37) ? q : (double)val[i];
    const double sm = shfl_sum(x);
    if (lane == 0) red[warp][i] = sm;
  }
  __syncthreads();
  if (threadIdx.x < kAvgPartials) {
    double sm = 0.0;
    for (int wq = 0; wq < (bd >> 5); ++wq) sm += red[wq][threadIdx.x];
    out40[threadIdx.x] = sm;
  }
  __syncthreads();
}

// Single: each thread accumulates its voxels' values in its own shared-memory
// column across the block's chunks (FP64, or compensated FP32 pairs for the
// values of FP32 fields); the block folds the columns once, in FP64, into
// partials[block][40] (a fixed grid gives a fixed order).  Multi:
// per-chunk records in each cell's apart.
template <class R, bool MULTI>
__global__ void __launch_bounds__(256) k_commit(CellDev<R> c0, Work<R> w, double* partials) {
  extern __shared__ __align__(16) unsigned char smem_raw[];  // single: [kAvgPartials][256] 8-byte slots
  __shared__ CellDev<R> cs;
  __shared__ double red[8][kAvgPartials];
  __shared__ double chunk_sum[kAvgPartials];
  double* cols = reinterpret_cast<double*>(smem_raw);
  if constexpr (!MULTI) {
    for (int i = threadIdx.x; i < kAvgPartials * (int)blockDim.x; i += blockDim.x) cols[i] = 0.0;
  }
  for_items<R, MULTI>(c0, (c0.nvox + 255) / 256, w, cs, [&](const CellDev<R>& c, long long chunk) {
    commit_chunk<R, !MULTI>(c, chunk, chunk_sum, red, cols);
    if constexpr (MULTI) {
      if (threadIdx.x < kAvgPartials) c.apart[chunk * kAvgPartials + threadIdx.x] = chunk_sum[threadIdx.x];
      __syncthreads();
    }
  });
  if constexpr (!MULTI) {
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < kAvgPartials; i += nw) {
      const bool pair = sizeof(R) == 4 && i != 36 && i != 37;  // compensated FP32 (hi, lo) column
      double sm = 0.0;
      for (int k = lane; k < (int)blockDim.x; k += 32) {
        if (pair) {
          const float2 a = reinterpret_cast<const float2*>(cols)[i * blockDim.x + k];
          sm += (double)a.x + (double)a.y;
        } else {
          sm += cols[i * blockDim.x + k];
        }
      }
      sm = shfl_sum(sm);
      if (lane == 0) partials[(long long)blockIdx.x * kAvgPartials + i] = sm;
    }
  }
}

// The loading-history magnitudes of the error measure (cell scalars 18..21)
// after a committed increment whose averages are row[0..35] (T, M, <e>, <gamma>).
__device__ __forceinline__ void update_history(const double* row, double* scalars) {
  double n[4] = {0.0, 0.0, 0.0, 0.0};  // ||<e>||, ||T||, ||<gamma>||, ||M||
  for (int q = 0; q < 9; ++q) {
    n[0] += row[18 + q] * row[18 + q];
    n[1] += row[q] * row[q];
    n[2] += row[27 + q] * row[27 + q];
    n[3] += row[9 + q] * row[9 + q];
  }
  for (int a = 0; a < 4; ++a) scalars[18 + a] = fmax(scalars[18 + a], sqrt(n[a]));
}

// Sum of the commit partials in a fixed order, divided by the voxel count.
__global__ void k_reduce_avg(const double* partials, int nparts, double inv_nvox, double* out, double* scalars) {
  __shared__ double row[kAvgPartials];
  if (threadIdx.x < kAvgPartials) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += partials[(long long)b * kAvgPartials + threadIdx.x];
    out[threadIdx.x] = row[threadIdx.x] = s * inv_nvox;
  }
  __syncthreads();
  if (threadIdx.x == 0) update_history(row, scalars);
}

// One block per entry: the cell's chunk records in chunk order -> c.avg_out.
template <class R>
__global__ void k_reduce_avg_multi(Work<R> w) {
  __shared__ CellDev<R> cs;
  load_cell(cs, w.cells + w.act[blockIdx.x]);
  __syncthreads();
  __shared__ double row[kAvgPartials];
  if (threadIdx.x < kAvgPartials) {
    const long long n = (cs.nvox + 255) / 256;
    double s = 0.0;
    for (long long b = 0; b < n; ++b) s += cs.apart[b * kAvgPartials + threadIdx.x];
    cs.avg_out[threadIdx.x] = row[threadIdx.x] = s * cs.inv_nvox;
  }
  __syncthreads();
  if (threadIdx.x == 0) update_history(row, cs.tmean);
}

// Final-state fields in FP64: e, gamma from `src` (prev or elast), t = h_t + A e,
// m = h_m + B gamma (the history form of the converged stresses), p, q.
template <class R>
__global__ void k_fields(CellDev<R> c, const R* src, int src_stride, double* fe, double* fg,
                         double* ft, double* fm, double* fp, double* fq) {
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < c.nvox;
       v += (long long)gridDim.x * blockDim.x) {
    const R* s = src + v * src_stride;
    const R* hv = c.hist + v * 20;
    R e[9], g[9], t[9], m[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      e[q] = s[q];
      g[q] = s[9 + q];
    }
    const PhaseDev<R> P = c.phases[c.phase[v]];
    apply_A<R>(P.lam, P.mu, P.kap, e, t);
    apply_B<R>(P.alpha, P.beta, P.gamma, g, m);
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      if (fe) fe[v * 9 + q] = (double)e[q];
      if (fg) fg[v * 9 + q] = (double)g[q];
      if (ft) ft[v * 9 + q] = (double)(hv[q] + t[q]);
      if (fm) fm[v * 9 + q] = (double)(hv[9 + q] + m[q]);
    }
    if (fp) fp[v] = c.pq[2 * v];
    if (fq) fq[v] = c.pq[2 * v + 1];
  }
}

// ------------------------------------------------------------------ component: Algorithm 1
template <class R>
__global__ void __launch_bounds__(256) k_radial_return_points(
    long long count, const uint16_t* phase, const PhaseDev<R>* phases, const R* e, const R* g,
    const R* e_n, const R* g_n, const R* t_n, const R* m_n, const double* p_n, const double* q_n,
    R* t, R* m, double* p, double* q) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const PhaseDev<R> P = phases[phase[i]];
    R ee[9], gg[9], en[9], gn[9], ht[9], hm[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      ee[k] = e[i * 9 + k];
      gg[k] = g[i * 9 + k];
      en[k] = e_n[i * 9 + k];
      gn[k] = g_n[i * 9 + k];
    }
    // history form of eq. trial_stresses: h_t = t_n - A e_n, h_m = m_n - B gamma_n
    apply_A<R>(P.lam, P.mu, P.kap, en, ht);
    apply_B<R>(P.alpha, P.beta, P.gamma, gn, hm);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      ht[k] = t_n[i * 9 + k] - ht[k];
      hm[k] = m_n[i * 9 + k] - hm[k];
    }
    R tt[9], mm[9];
    double pp, qq;
    R ft, fm;
    radial_return<R>(P, ee, gg, ht, hm, p_n[i], q_n[i], tt, mm, pp, qq, ft, fm);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      t[i * 9 + k] = tt[k];
      m[i * 9 + k] = mm[k];
    }
    p[i] = pp;
    q[i] = qq;
  }
}

// ------------------------------------------------------------------ launchers

template <class R>
size_t smem_pass_a(int n1, int rows) { return PassASmem<R>(n1, rows).total; }

constexpr size_t kCommitSmem = (size_t)kAvgPartials * 256 * sizeof(double);  // single-cell commit columns

// Raise each kernel's dynamic shared-memory limit to what its static shared
// memory leaves of the opt-in maximum (at least kSmemBudget).
template <class R>
static cudaError_t set_smem_attrs() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  // tiles: kernels whose tiles may take up to kSmemBudget (their static shared
  // memory must fit the reserve)
  auto raise = [&](const void* fn, bool tiles = true) {
    if (e != cudaSuccess) return;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return;
    if (tiles && fa.sharedSizeBytes > kSmemStaticReserve) {
      e = cudaErrorInvalidValue;
      return;
    }
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(kSmemOptin - fa.sharedSizeBytes));
  };
  raise((const void*)k_fft_y<R, -1, false, 0>);
  raise((const void*)k_fft_y<R, +1, false, 0>);
  raise((const void*)k_fft_y<R, -1, false, 128>);
  raise((const void*)k_fft_y<R, +1, false, 128>);
  raise((const void*)k_fft_y<R, -1, false, 256>);
  raise((const void*)k_fft_y<R, +1, false, 256>);
  raise((const void*)k_fft_y<R, -1, true, 0>);
  raise((const void*)k_fft_y<R, +1, true, 0>);
  raise((const void*)k_green_z<R, false, 0>);
  raise((const void*)k_green_z<R, false, 128>);
  raise((const void*)k_green_z<R, false, 256>);
  raise((const void*)k_green_z<R, true, 0>);
  raise((const void*)k_pass_a<R, kIter, false>);
  raise((const void*)k_pass_a<R, kStart, false>);
  raise((const void*)k_pass_a<R, kXFwd, false>);
  raise((const void*)k_pass_a<R, kXInv, false>);
  raise((const void*)k_pass_a<R, kIter, true>);
  raise((const void*)k_pass_a<R, kStart, true>);
  raise((const void*)k_commit<R, false>, false);
  if (e == cudaSuccess) done = true;
  return e;
}

template <class R>
int grid_for(const void* fn, int threads, size_t smem, long long work, int nsm) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (per_sm < 1) per_sm = 1;
  long long g = (long long)per_sm * nsm;
  if (work < g) g = work;
  if (g < 1) g = 1;
  return (int)g;
}

template <class R>
cudaError_t launch_fft_y(const LaunchCfg& L, const CellDev<R>& c, int dir, cudaStream_t st) {
  cudaError_t e = set_smem_attrs<R>();
  if (e != cudaSuccess) return e;
  if (c.n2 > 1) {
    const size_t sm = smem_line_pass<R>(c.n2);
    if (dir < 0) {
      if (c.n2 == 256) k_fft_y<R, -1, false, 256><<<L.grid_y, kThreadsYZ, sm, st>>>(c, Work<R>{});
      else if (c.n2 == 128) k_fft_y<R, -1, false, 128><<<L.grid_y, kThreadsYZ, sm, st>>>(c, Work<R>{});
      else k_fft_y<R, -1, false, 0><<<L.grid_y, kThreadsYZ, sm, st>>>(c, Work<R>{});
    } else {
      if (c.n2 == 256) k_fft_y<R, +1, false, 256><<<L.grid_y, kThreadsYZ, sm, st>>>(c, Work<R>{});
      else if (c.n2 == 128) k_fft_y<R, +1, false, 128><<<L.grid_y, kThreadsYZ, sm, st>>>(c, Work<R>{});
      else k_fft_y<R, +1, false, 0><<<L.grid_y, kThreadsYZ, sm, st>>>(c, Work<R>{});
    }
  }
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_green_z(const LaunchCfg& L, const CellDev<R>& c, cudaStream_t st) {
  cudaError_t e = set_smem_attrs<R>();
  if (e != cudaSuccess) return e;
  const size_t sm = smem_line_pass<R>(c.n3);
  if (c.n3 == 256) k_green_z<R, false, 256><<<L.grid_z, kThreadsYZ, sm, st>>>(c, Work<R>{});
  else if (c.n3 == 128) k_green_z<R, false, 128><<<L.grid_z, kThreadsYZ, sm, st>>>(c, Work<R>{});
  else k_green_z<R, false, 0><<<L.grid_z, kThreadsYZ, sm, st>>>(c, Work<R>{});
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_pass_a_iter(const LaunchCfg& L, const CellDev<R>& c, double* partials,
                               cudaStream_t st) {
  cudaError_t e = set_smem_attrs<R>();
  if (e != cudaSuccess) return e;
  k_pass_a<R, kIter, false><<<L.grid_a, kThreads, smem_pass_a<R>(c.n1, c.rows_a), st>>>(
      c, Work<R>{}, partials, nullptr, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_reduce_err(const LaunchCfg& L, const CellDev<R>& c, const double* partials,
                              int err_kind, double* err_out, cudaStream_t st) {
  k_reduce_err<R><<<1, 256, 0, st>>>(c, partials, L.grid_a, err_kind, err_out);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_reduce_err_loop(const LaunchCfg& L, const CellDev<R>& c, const double* partials, int err_kind,
                                   double* err_out, double tol, int max_iter, double div_limit, int stag,
                                   int adapt, cudaGraphConditionalHandle handle, cudaStream_t st) {
  k_reduce_err_loop<R><<<1, 256, 0, st>>>(c, partials, L.grid_a, err_kind, err_out, tol, max_iter, div_limit,
                                          stag, adapt, handle);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_iteration(const LaunchCfg& L, const CellDev<R>& c, double* partials,
                             double* err_out, int err_kind, cudaStream_t st) {
  cudaError_t e;
  if ((e = launch_fft_y<R>(L, c, -1, st)) != cudaSuccess) return e;
  if ((e = launch_green_z<R>(L, c, st)) != cudaSuccess) return e;
  if ((e = launch_fft_y<R>(L, c, +1, st)) != cudaSuccess) return e;
  if ((e = launch_pass_a_iter<R>(L, c, partials, st)) != cudaSuccess) return e;
  return launch_reduce_err<R>(L, c, partials, err_kind, err_out, st);
}

template <class R>
cudaError_t launch_start(const LaunchCfg& L, const CellDev<R>& c, int first, cudaStream_t st) {
  cudaError_t e = set_smem_attrs<R>();
  if (e != cudaSuccess) return e;
  if (first) k_init<R, false><<<L.grid_v, 256, 0, st>>>(c, Work<R>{});
  k_pass_a<R, kStart, false><<<L.grid_a, kThreads, smem_pass_a<R>(c.n1, c.rows_a), st>>>(
      c, Work<R>{}, nullptr, nullptr, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_commit(const LaunchCfg& L, const CellDev<R>& c, double* partials, double* avg_out,
                          cudaStream_t st) {
  k_commit<R, false><<<L.grid_v, 256, kCommitSmem, st>>>(c, Work<R>{}, partials);
  k_reduce_avg<<<1, 64, 0, st>>>(partials, L.grid_v, c.inv_nvox, avg_out, c.tmean);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ multi-cell launches
template <class R>
cudaError_t launch_multi_iteration(const MultiCfg<R>& m, cudaStream_t st) {
  cudaError_t e = set_smem_attrs<R>();
  if (e != cudaSuccess) return e;
  if (m.items_y > 0)
    k_fft_y<R, -1, true, 0><<<m.grid_y, kThreadsYZ, m.smem_y, st>>>(CellDev<R>{}, m.wy);
  if (m.items_z > 0)
    k_green_z<R, true, 0><<<m.grid_z, kThreadsYZ, m.smem_z, st>>>(CellDev<R>{}, m.wz);
  if (m.items_y > 0)
    k_fft_y<R, +1, true, 0><<<m.grid_y, kThreadsYZ, m.smem_y, st>>>(CellDev<R>{}, m.wy);
  if (m.items_a > 0)
    k_pass_a<R, kIter, true><<<m.grid_a, kThreads, m.smem_a, st>>>(CellDev<R>{}, m.wa, nullptr, nullptr,
                                                                    nullptr, nullptr, nullptr);
  if (m.wa.n_act > 0) k_reduce_err_multi<R><<<m.wa.n_act, 256, 0, st>>>(m.wa);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_multi_start(const MultiCfg<R>& m, cudaStream_t st) {
  cudaError_t e = set_smem_attrs<R>();
  if (e != cudaSuccess) return e;
  if (m.items_v0 > 0) k_init<R, true><<<m.grid_v0, 256, 0, st>>>(CellDev<R>{}, m.wv0);
  if (m.items_s > 0)
    k_pass_a<R, kStart, true><<<m.grid_s, kThreads, m.smem_a, st>>>(CellDev<R>{}, m.ws, nullptr, nullptr,
                                                                     nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_multi_commit(const MultiCfg<R>& m, cudaStream_t st) {
  if (m.items_v > 0) k_commit<R, true><<<m.grid_v, 256, 0, st>>>(CellDev<R>{}, m.wv, nullptr);
  if (m.wv.n_act > 0) k_reduce_avg_multi<R><<<m.wv.n_act, 64, 0, st>>>(m.wv);
  return cudaGetLastError();
}

template <class R>
void multi_grids(MultiCfg<R>& m, int nsm) {
  set_smem_attrs<R>();
  m.grid_y = grid_for<R>((const void*)k_fft_y<R, -1, true, 0>, kThreadsYZ, m.smem_y, m.items_y, nsm);
  m.grid_z = grid_for<R>((const void*)k_green_z<R, true, 0>, kThreadsYZ, m.smem_z, m.items_z, nsm);
  m.grid_a = grid_for<R>((const void*)k_pass_a<R, kIter, true>, kThreads, m.smem_a, m.items_a, nsm);
  m.grid_s = grid_for<R>((const void*)k_pass_a<R, kStart, true>, kThreads, m.smem_a, m.items_s, nsm);
  long long g = m.items_v < 8ll * nsm ? m.items_v : 8ll * nsm;
  m.grid_v = (int)(g > 0 ? g : 1);
  g = m.items_v0 < 8ll * nsm ? m.items_v0 : 8ll * nsm;
  m.grid_v0 = (int)(g > 0 ? g : 1);
}

template <class R>
cudaError_t launch_fields(const LaunchCfg& L, const CellDev<R>& c, int from_elast, double* fe,
                          double* fg, double* ft, double* fm, double* fp, double* fq, cudaStream_t st) {
  const R* src = from_elast ? c.elast : c.prev;
  const int stride = from_elast ? 18 : 20;
  k_fields<R><<<L.grid_v, 256, 0, st>>>(c, src, stride, fe, fg, ft, fm, fp, fq);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_green_apply(const LaunchCfg& L, const CellDev<R>& c, const R* tau, const R* mu,
                               R* e_out, R* g_out, cudaStream_t st, int* ctl, int nsm) {
  cudaError_t e = set_smem_attrs<R>();
  if (e != cudaSuccess) return e;
  const size_t sa = smem_pass_a<R>(c.n1, c.rows_a);
  k_pass_a<R, kXFwd, false><<<L.grid_a, kThreads, sa, st>>>(c, Work<R>{}, nullptr, tau, mu, nullptr, nullptr);
  bool fused = false;
  if constexpr (sizeof(R) == 4) {
    if (ctl) {
      fused = true;
      if ((e = launch_spectral(c, ctl, nsm, st)) != cudaSuccess) return e;
    }
  }
  if (!fused) {
    if (c.n2 > 1) k_fft_y<R, -1, false, 0><<<L.grid_y, kThreadsYZ, smem_line_pass<R>(c.n2), st>>>(c, Work<R>{});
    k_green_z<R, false, 0><<<L.grid_z, kThreadsYZ, smem_line_pass<R>(c.n3), st>>>(c, Work<R>{});
    if (c.n2 > 1) k_fft_y<R, +1, false, 0><<<L.grid_y, kThreadsYZ, smem_line_pass<R>(c.n2), st>>>(c, Work<R>{});
  }
  k_pass_a<R, kXInv, false><<<L.grid_a, kThreads, sa, st>>>(c, Work<R>{}, nullptr, nullptr, nullptr, e_out, g_out);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_radial_return(int nsm, long long count, const uint16_t* phase,
                                 const PhaseDev<R>* phases, const R* e, const R* g, const R* e_n,
                                 const R* g_n, const R* t_n, const R* m_n, const double* p_n,
                                 const double* q_n, R* t, R* m, double* p, double* q,
                                 cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  long long blocks = (count + 255) / 256;
  if (blocks > 8ll * nsm) blocks = 8ll * nsm;
  k_radial_return_points<R><<<(int)blocks, 256, 0, st>>>(count, phase, phases, e, g, e_n, g_n, t_n, m_n,
                                                          p_n, q_n, t, m, p, q);
  return cudaGetLastError();
}

// Element-wise precision conversion of device state (cells moving between
// the FP32 and FP64 engines).
template <class S, class D>
__global__ void k_convert(const S* __restrict__ src, D* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (D)src[i];
}

template <class S, class D>
cudaError_t launch_convert(const S* src, D* dst, long long n, int nsm, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  long long blocks = (n + 255) / 256;
  if (blocks > 8ll * nsm) blocks = 8ll * nsm;
  k_convert<S, D><<<(int)blocks, 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}
template cudaError_t launch_convert<float, double>(const float*, double*, long long, int, cudaStream_t);
template cudaError_t launch_convert<double, float>(const double*, float*, long long, int, cudaStream_t);

template <class R>
LaunchCfg make_launch_cfg(const CellDev<R>& c, int nsm, int rows_wanted) {
  set_smem_attrs<R>();
  LaunchCfg L;
  // rows per pass-A item: about 256 voxels per block (or as asked), within the
  // shared-memory budget
  int rows = rows_wanted > 0 ? rows_wanted : (c.n1 >= 256 ? 1 : 256 / c.n1);
  while (rows > 1 && smem_pass_a<R>(c.n1, rows) > kSmemBudget) rows /= 2;
  if ((long long)rows > (long long)c.n2 * c.n3) rows = (int)((long long)c.n2 * c.n3);
  L.rows = rows;
  const long long nrows = (long long)c.n2 * c.n3;
  const long long items = (nrows + rows - 1) / rows;
  L.items_a = items;
  L.grid_a = grid_for<R>((const void*)k_pass_a<R, kIter, false>, kThreads, smem_pass_a<R>(c.n1, rows), items,
                         nsm);
  const void* fy = c.n2 == 256   ? (const void*)k_fft_y<R, -1, false, 256>
                   : c.n2 == 128 ? (const void*)k_fft_y<R, -1, false, 128>
                                 : (const void*)k_fft_y<R, -1, false, 0>;
  const void* fz = c.n3 == 256   ? (const void*)k_green_z<R, false, 256>
                   : c.n3 == 128 ? (const void*)k_green_z<R, false, 128>
                                 : (const void*)k_green_z<R, false, 0>;
  L.grid_y = grid_for<R>(fy, kThreadsYZ, smem_line_pass<R>(c.n2), tiles_y(c), nsm);
  L.grid_z = grid_for<R>(fz, kThreadsYZ, smem_line_pass<R>(c.n3), tiles_z(c), nsm);
  long long vb = (c.nvox + 255) / 256;
  L.grid_v = (int)(vb < 4ll * nsm ? vb : 4ll * nsm);
  return L;
}

template <class R>
bool sizes_fit(int n1, int n2, int n3) {
  return smem_pass_a<R>(n1, 1) <= kSmemBudget && smem_line_pass<R>(n2) <= kSmemBudget &&
         smem_line_pass<R>(n3) <= kSmemBudget;
}

#define MP_INSTANTIATE(R)                                                                            \
  template cudaError_t launch_fft_y<R>(const LaunchCfg&, const CellDev<R>&, int, cudaStream_t);       \
  template cudaError_t launch_green_z<R>(const LaunchCfg&, const CellDev<R>&, cudaStream_t);          \
  template cudaError_t launch_pass_a_iter<R>(const LaunchCfg&, const CellDev<R>&, double*, cudaStream_t); \
  template cudaError_t launch_reduce_err_loop<R>(const LaunchCfg&, const CellDev<R>&, const double*, int, \
                                                 double*, double, int, double, int, int,             \
                                                 cudaGraphConditionalHandle, cudaStream_t);          \
  template cudaError_t launch_reduce_err<R>(const LaunchCfg&, const CellDev<R>&, const double*, int,  \
                                            double*, cudaStream_t);                                  \
  template cudaError_t launch_iteration<R>(const LaunchCfg&, const CellDev<R>&, double*, double*, int, \
                                           cudaStream_t);                                            \
  template cudaError_t launch_start<R>(const LaunchCfg&, const CellDev<R>&, int, cudaStream_t);       \
  template cudaError_t launch_commit<R>(const LaunchCfg&, const CellDev<R>&, double*, double*,        \
                                        cudaStream_t);                                               \
  template cudaError_t launch_multi_iteration<R>(const MultiCfg<R>&, cudaStream_t);                   \
  template cudaError_t launch_multi_start<R>(const MultiCfg<R>&, cudaStream_t);                       \
  template cudaError_t launch_multi_commit<R>(const MultiCfg<R>&, cudaStream_t);                      \
  template void multi_grids<R>(MultiCfg<R>&, int);                                                   \
  template size_t smem_pass_a<R>(int, int);                                                          \
  template size_t smem_line_pass<R>(int);                                                            \
  template cudaError_t launch_fields<R>(const LaunchCfg&, const CellDev<R>&, int, double*, double*,   \
                                        double*, double*, double*, double*, cudaStream_t);           \
  template cudaError_t launch_green_apply<R>(const LaunchCfg&, const CellDev<R>&, const R*, const R*,  \
                                             R*, R*, cudaStream_t, int*, int);                       \
  template cudaError_t launch_radial_return<R>(int, long long, const uint16_t*, const PhaseDev<R>*,   \
                                               const R*, const R*, const R*, const R*, const R*,      \
                                               const R*, const double*, const double*, R*, R*,        \
                                               double*, double*, cudaStream_t);                       \
  template LaunchCfg make_launch_cfg<R>(const CellDev<R>&, int, int);                                  \
  template bool sizes_fit<R>(int, int, int);

MP_INSTANTIATE(float)
MP_INSTANTIATE(double)

}  // namespace mp
