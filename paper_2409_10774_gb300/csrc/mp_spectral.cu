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
// Each item is one column of 18 lines x 256 points (144-byte chunks, one per
// point); its 288 threads are (line c, butterfly j), 18 x 16.  A block keeps
// two column tiles in shared memory: the next item's column is copied in
// (16-byte asynchronous copies) while the current one is transformed.  The
// 256-point transform is two radix-16 Stockham stages in place on the tile,
// the second with the twiddles W_256^(r j); the Y items store their result to
// global memory from registers, the Z items keep it in the tile for the Green
// operator and the inverse transform.
#include "mp_fft.cuh"
#include "mp_green.cuh"
#include "mp_kernels.cuh"

namespace mp {

namespace {

constexpr int kN = 256;            // y and z lengths handled here
constexpr int kLines = 18;         // components per spectral point
constexpr int kSpecThreads = 288;  // 18 lines x 16 butterflies
constexpr int kPhaseItems = kN;    // items per phase and plane (z or ky values)
constexpr int kTile = kN * kLines; // complex values of one column tile
constexpr int kPieces = kN * kLines * 8 / 16;  // 16-byte pieces of a tile

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

__device__ __forceinline__ void cp_async_cg16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void stcg(cpx<float>* p, cpx<float> v) {
  __stcg(reinterpret_cast<float2*>(p), make_float2(v.x, v.y));
}

// One work item: phase (0 = Y forward, 1 = Z with the Green operator, 2 = Y
// inverse) of plane g (kx = g) at position idx (z for the Y phases, ky for Z).
struct Item {
  int phase, g, idx;
  bool valid;
};

__device__ __forceinline__ Item decode(long long it, int KX) {
  // super-step t holds, interleaved, Y forward of plane t, Z of plane t - 1
  // and Y inverse of plane t - 2
  constexpr long long per_step = 3ll * kPhaseItems;
  Item r;
  const long long t = it / per_step;
  const int rem = (int)(it - t * per_step);
  r.phase = rem % 3;
  r.idx = rem / 3;
  r.g = (int)t - r.phase;
  r.valid = r.g >= 0 && r.g < KX;
  return r;
}

// The column of an item: first complex value of line 0 and the stride
// between its points (complex units).
__device__ __forceinline__ cpx<float>* column(const CellDev<float>& c, const Item& q, long long& stride) {
  if (q.phase == 1) {
    stride = (long long)c.n2 * c.kx * kLines;
    return c.spec + ((long long)q.idx * c.kx + q.g) * kLines;
  }
  stride = (long long)c.kx * kLines;
  return c.spec + ((long long)q.idx * c.n2 * c.kx + q.g) * kLines;
}

// Asynchronous copy of an item's column into a shared-memory tile laid out
// as the spectrum stores a point ([point][18 lines], 144 bytes apart): 16-byte
// pieces, several per thread, completion through the thread's copy groups.
__device__ __forceinline__ void issue_column(const CellDev<float>& c, const Item& q, cpx<float>* tile) {
  long long stride;
  const cpx<float>* col = column(c, q, stride);
  const char* src = reinterpret_cast<const char*>(col);
  char* dst = reinterpret_cast<char*>(tile);
  for (int k = threadIdx.x; k < kPieces; k += kSpecThreads) {
    const int pt = k / 9, piece = k - pt * 9;
    cp_async_cg16(dst + pt * 144 + piece * 16, src + (long long)pt * stride * 8 + piece * 16);
  }
}

// Stage one of a 256-point transform on the tile: thread (c, j) takes points
// j + 16 r (r < 16) of line c, forms their 16-point DFT and, once every
// thread has read its inputs, writes output r to position 16 j + r.
template <int DIR>
__device__ __forceinline__ void stage1(cpx<float>* w, int c, int j) {
  cpx<float> v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = w[(j + 16 * r) * kLines + c];
  dft16<float, DIR>(v);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) w[(16 * j + r) * kLines + c] = v[r];
  __syncthreads();
}

// Stage two: thread (c, j) takes positions 16 r + j of line c, multiplies
// position r by W_256^(r j) (conjugated for the inverse) and forms the 16-point
// DFT; output k is point j + 16 k of the transformed line.
template <int DIR>
__device__ __forceinline__ void stage2(const cpx<float>* w, const cpx<float>* tw, int c, int j, cpx<float> (&v)[16]) {
  v[0] = w[j * kLines + c];
#pragma unroll
  for (int r = 1; r < 16; ++r) v[r] = cmul(w[(16 * r + j) * kLines + c], twiddle<float, DIR>(tw, r * j));
  dft16<float, DIR>(v);
}

template <int DIR>
__device__ __forceinline__ void y_compute(const CellDev<float>& c, const Item& q, cpx<float>* w, const cpx<float>* tw,
                                          int line, int j) {
  long long stride;
  cpx<float>* col = column(c, q, stride) + line;
  stage1<DIR>(w, line, j);
  cpx<float> v[16];
  stage2<DIR>(w, tw, line, j, v);
#pragma unroll
  for (int k = 0; k < 16; ++k) stcg(col + (long long)(j + 16 * k) * stride, v[k]);
}

__device__ __forceinline__ void z_compute(const CellDev<float>& c, const Item& q, cpx<float>* w, const cpx<float>* tw,
                                          int line, int j) {
  long long stride;
  cpx<float>* col = column(c, q, stride) + line;
  const int ky = q.idx, kx = q.g;
  stage1<-1>(w, line, j);
  {
    cpx<float> v[16];
    stage2<-1>(w, tw, line, j, v);
    __syncthreads();  // every thread has read its stage-two inputs
#pragma unroll
    for (int k = 0; k < 16; ++k) w[(j + 16 * k) * kLines + line] = v[k];
  }
  __syncthreads();
  // Green operator at each point kz of the column (one thread per point)
  const int kz = threadIdx.x;
  if (kz < kN) {
    cpx<float>* pt = w + kz * kLines;
    const bool nyq = (ky == c.n2 / 2) || (kz == kN / 2);
    const bool zero = (kx == 0 && ky == 0 && kz == 0);
    if (nyq || zero) {
#pragma unroll
      for (int r = 0; r < kLines; ++r) pt[r] = cmake<float>(0.f, 0.f);
    } else {
      const float x1 = c.two_pi_over_L[0] * (float)kx;
      const float x2 = c.two_pi_over_L[1] * (float)(ky <= c.n2 / 2 ? ky : ky - c.n2);
      const float x3 = c.two_pi_over_L[2] * (float)(kz <= kN / 2 ? kz : kz - kN);
      green_point<float>(c.ref, x1, x2, x3, pt, (float)c.inv_nvox);
    }
  }
  __syncthreads();
  stage1<+1>(w, line, j);
  cpx<float> v[16];
  stage2<+1>(w, tw, line, j, v);
#pragma unroll
  for (int k = 0; k < 16; ++k) stcg(col + (long long)(j + 16 * k) * stride, v[k]);
}

// ctl[0]: work-queue head; ctl[1 + p * KX + g]: finished items of phase p
// (0 = Y forward, 1 = Z) of plane g.  Zeroed before every launch.
//
// Each block keeps two column tiles: while it transforms the current item in
// one, the next item's column is already being copied into the other (when
// that item's inputs are complete; otherwise the copy is issued after the
// current item, which may be one the next item waits for).
__global__ void __launch_bounds__(kSpecThreads, 3) k_spectral(CellDev<float> c, int* ctl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<float>* tiles = reinterpret_cast<cpx<float>*>(smem_raw);  // [2][kTile]
  cpx<float>* tw = tiles + 2 * kTile;                            // W_256^k (the y and z tables coincide)
  __shared__ long long item_s;
  __shared__ int ready_s;
  const int line = threadIdx.x % kLines, j = threadIdx.x / kLines;
  for (int k = threadIdx.x; k < kN; k += blockDim.x) tw[k] = c.py.tw[k];
  const int KX = c.kx;
  const long long total = ((long long)KX + 2) * 3 * kPhaseItems;
  int* status = c.status;
  auto dep_counter = [&](const Item& q) { return &ctl[1 + (q.phase - 1) * KX + q.g]; };

  // first item: fetch, wait for its inputs, copy
  if (threadIdx.x == 0) {
    long long it;
    Item q;
    do {  // skip the empty slots of the first super-steps
      it = atomicAdd(&ctl[0], 1);
      q = decode(it, KX);
    } while (it < total && !q.valid);
    bool ok = true;
    if (it < total && q.phase > 0) {
      ok = wait_count(dep_counter(q), kPhaseItems, status);
      if (!ok) atomicOr(status, 1);
      __threadfence();
    }
    item_s = ok ? it : total;
  }
  __syncthreads();
  long long cur = item_s;
  int b = 0;
  if (cur < total) issue_column(c, decode(cur, KX), tiles);
  cp_async_commit();
  while (cur < total) {
    const Item q = decode(cur, KX);
    // next item: fetch it and, when its inputs are complete, start its copy
    if (threadIdx.x == 0) {
      long long it;
      Item n;
      do {
        it = atomicAdd(&ctl[0], 1);
        n = decode(it, KX);
      } while (it < total && !n.valid);
      int ready = 1;
      if (it < total && n.phase > 0) {
        ready = ld_acquire_gpu(dep_counter(n)) >= kPhaseItems;
        if (ready) __threadfence();
      }
      item_s = it;
      ready_s = ready;
    }
    __syncthreads();
    const long long nxt = item_s;
    const bool ready = ready_s != 0;
    cpx<float>* wcur = tiles + b * kTile;
    cpx<float>* wnxt = tiles + (b ^ 1) * kTile;
    if (nxt < total && ready) issue_column(c, decode(nxt, KX), wnxt);
    cp_async_commit();
    cp_async_wait<1>();  // the current item's copy (the older group)
    __syncthreads();
    if (q.phase == 0) y_compute<-1>(c, q, wcur, tw, line, j);
    else if (q.phase == 1) z_compute(c, q, wcur, tw, line, j);
    else y_compute<+1>(c, q, wcur, tw, line, j);
    __syncthreads();  // the item's stores are issued and its tile is free
    if (q.phase < 2 && threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&ctl[1 + q.phase * KX + q.g], 1);
    }
    if (nxt < total && !ready) {
      // the next item waits (bounded) for its inputs, then copies
      if (threadIdx.x == 0) {
        const Item n = decode(nxt, KX);
        const bool ok = wait_count(dep_counter(n), kPhaseItems, status);
        if (!ok) atomicOr(status, 1);
        __threadfence();
      }
      __syncthreads();
      issue_column(c, decode(nxt, KX), wnxt);
      cp_async_commit();
    }
    cur = nxt;
    b ^= 1;
  }
  cp_async_wait<0>();
}

}  // namespace

size_t spectral_ctl_ints(int kx) { return 1 + 2 * (size_t)kx; }

bool spectral_fused_ok(const CellDev<float>& c) {
  return c.n1 >= 2 && c.n2 == kN && c.n3 == kN && c.kx == c.n1 / 2;
}

constexpr size_t kSpecSmem = (2 * (size_t)kTile + kN) * sizeof(cpx<float>);

cudaError_t launch_spectral(const CellDev<float>& c, int* ctl, int nsm, cudaStream_t st) {
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_spectral, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSpecSmem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spectral, kSpecThreads, kSpecSmem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
  }
  cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(int) * spectral_ctl_ints(c.kx), st);
  if (e != cudaSuccess) return e;
  k_spectral<<<per_sm * nsm, kSpecThreads, kSpecSmem, st>>>(c, ctl);
  return cudaGetLastError();
}

}  // namespace mp
