// Fused spectral pass of one fixed-point iteration (sm_103a, FP32 fields):
// y forward, z forward, Green operator (eq. micropolar_LippmannSchwinger_iteration),
// z inverse and y inverse of the 18-component half spectrum, for cells whose
// y and z lengths are 256.
//
// The three separate column passes (y forward, z + Green + z, y inverse) each
// stream the whole 1.2 GB spectrum of a 256^3 cell through HBM.  Here one
// persistent kernel runs them as three phases per kx column-plane (all y and
// z of one kx: 256 x 256 points x 18 components, 9.4 MB in FP32) and takes
// its work items from one sequence in the order
//     Y-forward(g), Z(g - 2), Y-inverse(g - 4),  g = 0, 1, 2, ...
// so that a plane is read from HBM by its Y-forward items, revisited by its Z
// and Y-inverse items while it is still in L2 (about five planes, 47 MB, are
// live at a time), and written back once.  A Z item of plane g waits until
// every Y-forward item of g has finished, a Y-inverse item until every Z item
// of g has.  Block b takes positions b, b + G, b + 2 G, ... of the sequence
// (G blocks, all resident at once: a cooperative launch); each item waits
// only on items at earlier positions, which resident blocks reach first, so
// the waits always end.  They are bounded all the same: a wait that gives up
// records status bit 1 and the item is skipped (the host reports
// MP_E_TIMEOUT).
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
constexpr int kPieces = kN * kLines * 8 / 16;  // 16-byte pieces of a tile (9 per point)

__device__ __forceinline__ int ld_acquire_gpu(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void cp_async_cg16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
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

// Super-steps between the phases of one plane: the items a phase waits for
// were queued kLag super-steps (kLag * 768 items) earlier, well beyond the
// items the running blocks hold at once, so those are normally finished.
constexpr int kLag = 2;

__device__ __forceinline__ Item decode(long long it, int KX) {
  // super-step t holds, interleaved, Y forward of plane t, Z of plane
  // t - kLag and Y inverse of plane t - 2 kLag
  constexpr long long per_step = 3ll * kPhaseItems;
  Item r;
  const long long t = it / per_step;
  const int rem = (int)(it - t * per_step);
  r.phase = rem % 3;
  r.idx = rem / 3;
  r.g = (int)t - kLag * r.phase;
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

// ------------------------------------------------------------------ pipeline
// Warp-specialised blocks: warps 0-8 (288 threads) transform tiles, warp 9
// fetches work.  The producer warp takes the next item from the queue, waits
// (bounded) until the items it depends on have finished, and copies its
// column into a free tile slot with 16-byte asynchronous copies whose
// completion is signalled on the slot's "full" mbarrier; the consumer warps
// wait on that barrier, transform the tile, store their results, signal the
// item's completion counter and release the slot through its "empty" barrier.
// Consumers never wait for the queue or for other blocks, so their barriers
// only order work within the tile.
constexpr int kStages = 3;
constexpr int kConsumers = kSpecThreads;           // 9 warps
constexpr int kBlock = kSpecThreads + 32;          // + the producer warp
constexpr int kTimeoutSpins = 1 << 22;

struct SlotInfo {
  int phase, g, idx, last;  // last != 0: no more items for this block
};

__device__ __forceinline__ uint32_t sptr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sptr(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sptr(b)) : "memory");
}
// arrive on b once all of this thread's earlier cp.async copies are complete
__device__ __forceinline__ void mb_arrive_cp_async(uint64_t* b) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(sptr(b)) : "memory");
}
__device__ __forceinline__ bool mb_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(sptr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of b; gives up early once a failure is recorded.
__device__ __forceinline__ bool mb_wait(uint64_t* b, uint32_t parity, const int* status) {
  for (int i = 0; i < kTimeoutSpins; ++i) {
    if (mb_try(b, parity)) return true;
    if ((i & 255) == 255 && ld_acquire_gpu(status) != 0) return false;
    if (i > 256) __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ void consumer_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kConsumers) : "memory"); }

// The in-tile transforms of the consumers: the same stages as above with the
// consumers' named barrier in place of __syncthreads.
template <int DIR>
__device__ __forceinline__ void stage1_c(cpx<float>* w, int c, int j) {
  cpx<float> v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = w[(j + 16 * r) * kLines + c];
  dft16<float, DIR>(v);
  consumer_sync();
#pragma unroll
  for (int r = 0; r < 16; ++r) w[(16 * j + r) * kLines + c] = v[r];
  consumer_sync();
}

template <int DIR>
__device__ __forceinline__ void y_consume(const CellDev<float>& c, const Item& q, cpx<float>* w, const cpx<float>* tw,
                                          int line, int j) {
  long long stride;
  cpx<float>* col = column(c, q, stride) + line;
  stage1_c<DIR>(w, line, j);
  cpx<float> v[16];
  stage2<DIR>(w, tw, line, j, v);
#pragma unroll
  for (int k = 0; k < 16; ++k) stcg(col + (long long)(j + 16 * k) * stride, v[k]);
}

__device__ __forceinline__ void z_consume(const CellDev<float>& c, const Item& q, cpx<float>* w, const cpx<float>* tw,
                                          int line, int j) {
  long long stride;
  cpx<float>* col = column(c, q, stride) + line;
  const int ky = q.idx, kx = q.g;
  stage1_c<-1>(w, line, j);
  {
    cpx<float> v[16];
    stage2<-1>(w, tw, line, j, v);
    consumer_sync();  // every consumer has read its stage-two inputs
#pragma unroll
    for (int k = 0; k < 16; ++k) w[(j + 16 * k) * kLines + line] = v[k];
  }
  consumer_sync();
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
  consumer_sync();
  stage1_c<+1>(w, line, j);
  cpx<float> v[16];
  stage2<+1>(w, tw, line, j, v);
#pragma unroll
  for (int k = 0; k < 16; ++k) stcg(col + (long long)(j + 16 * k) * stride, v[k]);
}

// ctl[0]: unused; ctl[1 + p * KX + g]: finished items of phase p (0 = Y
// forward, 1 = Z) of plane g; ctl[1 + 2 KX]: finished blocks.  Zero at launch
// (allocation, then the last block of every launch).
__global__ void __launch_bounds__(kBlock, 2) k_spectral(CellDev<float> c, int* ctl) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<float>* tiles = reinterpret_cast<cpx<float>*>(smem_raw);                 // [kStages][kTile]
  cpx<float>* tw = tiles + kStages * kTile;                                     // W_256^k (y and z alike)
  uint64_t* full = reinterpret_cast<uint64_t*>(tw + kN);                       // [kStages]
  uint64_t* empty = full + kStages;                                             // [kStages]
  SlotInfo* info = reinterpret_cast<SlotInfo*>(empty + kStages);               // [kStages]
  for (int k = threadIdx.x; k < kN; k += blockDim.x) tw[k] = c.py.tw[k];
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mb_init(&full[s], 33);  // the producer's 32 lanes once their copies have landed, + lane 0's slot info
      mb_init(&empty[s], 1);  // the consumers' leader, once the tile is free
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int KX = c.kx;
  const long long total = ((long long)KX + 2 * kLag) * 3 * kPhaseItems;
  int* status = c.status;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == kConsumers / 32) {
    // ---------------------------------------------------------------- producer
    // Static assignment: this block's items are queue positions b, b + G,
    // b + 2 G, ... (G blocks, all resident: cooperative launch).  Inputs are
    // checked ahead: lanes 0-7 read the completion counters of the block's
    // next eight items at once, so one round trip usually covers eight items.
    const long long G = gridDim.x;
    long long pos = blockIdx.x;
    long long ready_upto = -1;  // every position <= this one has its inputs complete
    for (long long k = 0;; ++k) {
      const int s = (int)(k % kStages);
      const uint32_t round = (uint32_t)(k / kStages);
      // the slot's previous item has been consumed
      if (round > 0 && !mb_wait(&empty[s], (round - 1) & 1u, status)) {
        if (lane == 0) atomicOr(status, 1);
        break;
      }
      while (pos < total && !decode(pos, KX).valid) pos += G;
      long long it = pos;
      if (it < total && it > ready_upto) {
        bool ok_wait = false;
        for (int spin = 0; spin < kTimeoutSpins; ++spin) {
          bool ok = true;
          if (lane < 8) {
            const long long p2 = it + lane * G;
            if (p2 < total) {
              const Item d = decode(p2, KX);
              if (d.valid && d.phase > 0) ok = ld_acquire_gpu(&ctl[1 + (d.phase - 1) * KX + d.g]) >= kPhaseItems;
            }
          }
          const unsigned m = __ballot_sync(0xffffffffu, ok) & 0xffu;
          const int prefix = __ffs(~m | 0x100u) - 1;  // ready items from `it` on
          if (prefix > 0) {
            ready_upto = it + (long long)(prefix - 1) * G;
            ok_wait = true;
            break;
          }
          if ((spin & 255) == 255 && ld_acquire_gpu(status) != 0) break;
          if (spin > 32) __nanosleep(128);
        }
        if (!ok_wait) {
          if (lane == 0) atomicOr(status, 1);
          it = total;
        }
      }
      const Item q = decode(it < total ? it : 0, KX);
      if (lane == 0) info[s] = SlotInfo{q.phase, q.g, q.idx, it >= total ? 1 : 0};
      __syncwarp();
      if (it < total) {
        long long stride;
        const char* src = reinterpret_cast<const char*>(column(c, q, stride));
        char* dst = reinterpret_cast<char*>(tiles + s * kTile);
        for (int p = lane; p < kPieces; p += 32) {
          const int pt = p / 9, piece = p - pt * 9;
          cp_async_cg16(dst + pt * 144 + piece * 16, src + (long long)pt * stride * 8 + piece * 16);
        }
      }
      if (lane == 0) mb_arrive(&full[s]);  // releases the slot info written above
      mb_arrive_cp_async(&full[s]);        // (an item-less slot completes at once)
      if (it >= total) break;
      pos += G;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else {
  // ------------------------------------------------------------------ consumers
  const int line = threadIdx.x % kLines, j = threadIdx.x / kLines;
  for (long long k = 0;; ++k) {
    const int s = (int)(k % kStages);
    const uint32_t round = (uint32_t)(k / kStages);
    if (!mb_wait(&full[s], round & 1u, status)) {
      if (threadIdx.x == 0) atomicOr(status, 1);
      break;
    }
    const SlotInfo si = info[s];
    if (si.last) break;
    Item q;
    q.phase = si.phase;
    q.g = si.g;
    q.idx = si.idx;
    q.valid = true;
    cpx<float>* w = tiles + s * kTile;
    if (q.phase == 0) y_consume<-1>(c, q, w, tw, line, j);
    else if (q.phase == 1) z_consume(c, q, w, tw, line, j);
    else y_consume<+1>(c, q, w, tw, line, j);
    consumer_sync();  // the item's stores are issued and its tile is read
    if (threadIdx.x == 0) {
      if (q.phase < 2) {
        __threadfence();
        atomicAdd(&ctl[1 + q.phase * KX + q.g], 1);
      }
      mb_arrive(&empty[s]);
    }
  }
  }
  // The last block to finish zeroes the queue and the completion counters
  // for the next launch (so a launch needs no preceding memset).
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ctl[1 + 2 * KX], 1) == (int)gridDim.x - 1) {
      for (int i = 0; i < 2 + 2 * KX; ++i) ctl[i] = 0;
      __threadfence();
    }
  }
}

}  // namespace

size_t spectral_ctl_ints(int kx) { return 2 + 2 * (size_t)kx; }

bool spectral_fused_ok(const CellDev<float>& c) {
  return c.n1 >= 2 && c.n2 == kN && c.n3 == kN && c.kx == c.n1 / 2;
}

constexpr size_t kSpecSmem = ((size_t)kStages * kTile + kN) * sizeof(cpx<float>) +
                             2 * kStages * sizeof(uint64_t) + kStages * sizeof(SlotInfo);

cudaError_t launch_spectral(const CellDev<float>& c, int* ctl, int nsm, cudaStream_t st) {
  static int per_sm = 0;
  if (per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_spectral, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSpecSmem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_spectral, kBlock, kSpecSmem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
  }
  // the blocks wait on one another's items: all must be resident at once
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(per_sm * nsm));
  cfg.blockDim = dim3(kBlock);
  cfg.dynamicSmemBytes = kSpecSmem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_spectral, c, ctl);
}

}  // namespace mp
