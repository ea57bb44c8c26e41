// Shared-memory Stockham FFT building blocks (sm_103a).  Transforms are
// unnormalised; the solver folds the 1 / (N1 N2 N3) of the inverse into the
// Green operator.
#pragma once

#include "mp_common.cuh"

namespace mp {

// DIR = -1: forward kernel exp(-2 pi i k n / M); DIR = +1: inverse.
template <class R, int DIR>
__device__ __forceinline__ cpx<R> twiddle(const cpx<R>* tw, int idx) {
  cpx<R> w = tw[idx];
  if (DIR > 0) w.y = -w.y;
  return w;
}

// multiply by DIR * i  (the quarter-turn W_4 = exp(DIR i pi / 2))
template <class R, int DIR>
__device__ __forceinline__ cpx<R> rot90(cpx<R> a) {
  return DIR < 0 ? cmake<R>(a.y, -a.x) : cmake<R>(-a.y, a.x);
}

template <class R, int DIR>
__device__ __forceinline__ void dft2(cpx<R>* v) {
  cpx<R> a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <class R, int DIR>
__device__ __forceinline__ void dft3(cpx<R>* v) {
  // W_3 = -1/2 + DIR i sqrt(3)/2
  const R half = R(0.5);
  const R s3 = R(0.86602540378443864676372317075294);
  cpx<R> a = v[0], t = cadd(v[1], v[2]), u = csub(v[1], v[2]);
  cpx<R> base = cmake<R>(a.x - half * t.x, a.y - half * t.y);
  cpx<R> r = rot90<R, DIR>(cscale(u, s3));
  v[0] = cadd(a, t);
  v[1] = cadd(base, r);
  v[2] = csub(base, r);
}

template <class R, int DIR>
__device__ __forceinline__ void dft4(cpx<R>* v) {
  cpx<R> t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
  cpx<R> t2 = cadd(v[1], v[3]), t3 = rot90<R, DIR>(csub(v[1], v[3]));
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}

template <class R, int DIR>
__device__ __forceinline__ void dft8(cpx<R>* v) {
  // split into even / odd 4-point DFTs, combine with W_8^k = exp(DIR 2 pi i k / 8)
  cpx<R> e[4] = {v[0], v[2], v[4], v[6]};
  cpx<R> o[4] = {v[1], v[3], v[5], v[7]};
  dft4<R, DIR>(e);
  dft4<R, DIR>(o);
  const R h = R(0.70710678118654752440084436210485);
  // W_8^1 = h (1 + DIR i), W_8^2 = DIR i, W_8^3 = h (-1 + DIR i)
  cpx<R> o1 = cmake<R>(h * (o[1].x - DIR * o[1].y), h * (o[1].y + DIR * o[1].x));
  cpx<R> o2 = rot90<R, DIR>(o[2]);
  cpx<R> o3 = cmake<R>(h * (-o[3].x - DIR * o[3].y), h * (-o[3].y + DIR * o[3].x));
  v[0] = cadd(e[0], o[0]);
  v[4] = csub(e[0], o[0]);
  v[1] = cadd(e[1], o1);
  v[5] = csub(e[1], o1);
  v[2] = cadd(e[2], o2);
  v[6] = csub(e[2], o2);
  v[3] = cadd(e[3], o3);
  v[7] = csub(e[3], o3);
}

// 16-point DFT as 4 x 4: 4-point DFTs over n1 of x[4 n1 + n2], twiddles
// W_16^(n2 k1), 4-point DFTs over n2; output index k1 + 4 k2.
template <class R, int DIR>
__device__ __forceinline__ void dft16(cpx<R>* v) {
  cpx<R> a[4][4];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    cpx<R> t[4] = {v[n2], v[4 + n2], v[8 + n2], v[12 + n2]};
    dft4<R, DIR>(t);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) a[n2][k1] = t[k1];
  }
  // W_16^m = cos(2 pi m / 16) + DIR i sin(2 pi m / 16), m = n2 k1 in {1, 2, 3, 4, 6, 9}
  const R c1 = R(0.92387953251128675612818318939679);  // cos(pi/8)
  const R s1 = R(0.38268343236508977172845998403040);  // sin(pi/8)
  const R h = R(0.70710678118654752440084436210485);
  auto rot = [&](cpx<R> x, R cr, R si) {  // x * (cr + DIR i si)
    return cmake<R>(x.x * cr - DIR * x.y * si, x.y * cr + DIR * x.x * si);
  };
  a[1][1] = rot(a[1][1], c1, s1);
  a[1][2] = rot(a[1][2], h, h);
  a[1][3] = rot(a[1][3], s1, c1);
  a[2][1] = rot(a[2][1], h, h);
  a[2][2] = rot90<R, DIR>(a[2][2]);
  a[2][3] = rot(a[2][3], -h, h);
  a[3][1] = rot(a[3][1], s1, c1);
  a[3][2] = rot(a[3][2], -h, h);
  a[3][3] = rot(a[3][3], -c1, -s1);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    cpx<R> t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
    dft4<R, DIR>(t);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
  }
}

// Tiles are stored component-interleaved ("AoS"): element (row rr, point n,
// component c) of a tile with `rows` rows of M points lives at
// base[(rr M + n) 18 + c], exactly as the spectral buffer stores a row.  A
// transform line is (rr, c), with stride 18 between its points.  Threads take
// (c, j, rr) with c fastest, so a warp reads and writes consecutive complex
// values: the stages are free of shared-memory bank conflicts and need no
// transposition on load or store.
//
// One Stockham stage of radix R (2, 3, 4, 8 or 16) with Ns = product of the radices already
// applied: butterfly j of a line reads points j + r M / R (r < R), multiplies
// point r by W_M^(r (j mod Ns) M / (Ns R)), takes the R-point DFT and writes
// output r to point (j / Ns) Ns R + (j mod Ns) + r Ns.  The last stage leaves
// natural order (no bit reversal).  The host orders radix-3 stages last, so
// only those divide by a non-power-of-two Ns.
// MAXR bounds the radices a kernel instantiates (8 keeps the 16-point
// butterfly's registers out of kernels that never use it).
template <class R, int DIR, int MAXR>
__device__ void stage_aos(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out, int rows, int M,
                          int radix, int Ns, const cpx<R>* __restrict__ tw, int tstride) {
  const int nb = M / radix;
  const int total = rows * nb * 18;
  const int tstep = M / (Ns * radix);
  const bool ns_pow2 = (Ns & (Ns - 1)) == 0;
  const int ns_sh = __ffs(Ns) - 1;
  const bool nb_pow2 = (nb & (nb - 1)) == 0;
  const int nb_sh = __ffs(nb) - 1;
  const int rs = M * 18;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int c = idx % 18;
    const int q = idx / 18;
    int rr = 0, j = q;
    if (rows > 1) {
      rr = nb_pow2 ? (q >> nb_sh) : (q / nb);
      j = q - rr * nb;
    }
    const int kk = ns_pow2 ? (j & (Ns - 1)) : (j % Ns);
    const int jq = ns_pow2 ? (j >> ns_sh) : (j / Ns);
    const cpx<R>* src = in + rr * rs + c;
    cpx<R> v[MAXR];
    v[0] = src[j * 18];
#pragma unroll
    for (int r = 1; r < MAXR; ++r) {
      if (r < radix) {
        cpx<R> x = src[(j + r * nb) * 18];
        const int e = r * kk * tstep;  // < M
        v[r] = e == 0 ? x : cmul(x, twiddle<R, DIR>(tw, e * tstride));
      }
    }
    switch (radix) {
      case 2: dft2<R, DIR>(v); break;
      case 3: dft3<R, DIR>(v); break;
      case 4: dft4<R, DIR>(v); break;
      case 8: dft8<R, DIR>(v); break;
      default:
        if constexpr (MAXR >= 16) dft16<R, DIR>(v);
        break;
    }
    cpx<R>* dst = out + rr * rs + c + (jq * Ns * radix + kk) * 18;
#pragma unroll
    for (int r = 0; r < MAXR; ++r) {
      if (r < radix) dst[r * Ns * 18] = v[r];
    }
  }
}

// The same stage with the radix, Ns, the line length M and the twiddle stride
// known at compile time (index arithmetic folds to shifts and constants, and
// only the one butterfly is instantiated).  LN lines are interleaved point by
// point (18 components of one column, or of several columns side by side).
template <class R, int DIR, int RADIX, int NS, int M, int TSTRIDE, int LN = 18>
__device__ __forceinline__ void stage_fixed(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out, int rows,
                                            const cpx<R>* __restrict__ tw) {
  constexpr int nb = M / RADIX;
  constexpr int tstep = M / (NS * RADIX);
  constexpr int rs = M * LN;
  const int total = rows * nb * LN;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int c = idx % LN;
    const int q = idx / LN;
    const int rr = q / nb, j = q % nb;
    const int kk = j % NS, jq = j / NS;
    const cpx<R>* src = in + rr * rs + c;
    cpx<R> v[RADIX];
    v[0] = src[j * LN];
#pragma unroll
    for (int r = 1; r < RADIX; ++r) {
      const cpx<R> x = src[(j + r * nb) * LN];
      v[r] = (NS == 1) ? x : cmul(x, twiddle<R, DIR>(tw, r * kk * tstep * TSTRIDE));
    }
    if constexpr (RADIX == 2) dft2<R, DIR>(v);
    else if constexpr (RADIX == 3) dft3<R, DIR>(v);
    else if constexpr (RADIX == 4) dft4<R, DIR>(v);
    else if constexpr (RADIX == 8) dft8<R, DIR>(v);
    else dft16<R, DIR>(v);
    cpx<R>* dst = out + rr * rs + c + (jq * NS * RADIX + kk) * LN;
#pragma unroll
    for (int r = 0; r < RADIX; ++r) dst[r * NS * LN] = v[r];
  }
}

// Transform every line of an AoS tile; data starts in b0, the result pointer
// (b0 or b1) is returned.  Ends with a barrier.  `tw`, when given, is a copy
// of the plan's twiddle table (e.g. in shared memory).
template <class R, int DIR, int MAXR>
__device__ cpx<R>* tile_fft(cpx<R>* b0, cpx<R>* b1, int rows, const AxisPlan<R>& p,
                            const cpx<R>* tw = nullptr) {
  cpx<R>* in = b0;
  cpx<R>* out = b1;
  int Ns = 1;
  const cpx<R>* table = tw ? tw : p.tw;
  for (int s = 0; s < p.nstages; ++s) {
    stage_aos<R, DIR, MAXR>(in, out, rows, p.m, p.radix[s], Ns, table, p.tstride);
    Ns *= p.radix[s];
    __syncthreads();
    cpx<R>* t = in;
    in = out;
    out = t;
  }
  return in;
}

// The x-axis transform inside pass A (twiddle stride 2: the table holds the
// N1 = 2 M roots).  Common lengths are unrolled at compile time (radix <= 8,
// radix 3 last, except 16 x 8 for M = 128 in FP32); others take tile_fft with
// the host's radix plan.
template <class R, int DIR>
__device__ cpx<R>* tile_fft_x(cpx<R>* b0, cpx<R>* b1, int rows, const AxisPlan<R>& p, const cpx<R>* tw) {
  auto sync_swap = [&]() {
    __syncthreads();
    cpx<R>* t = b0;
    b0 = b1;
    b1 = t;
  };
  switch (p.m) {
    case 256:
      stage_fixed<R, DIR, 8, 1, 256, 2>(b0, b1, rows, tw); sync_swap();
      stage_fixed<R, DIR, 8, 8, 256, 2>(b0, b1, rows, tw); sync_swap();
      stage_fixed<R, DIR, 4, 64, 256, 2>(b0, b1, rows, tw); sync_swap();
      return b0;
    case 128:
      if constexpr (sizeof(R) == 4) {
        // two stages (16 x 8): one shared-memory pass and one barrier fewer
        // (FP64 keeps three: its radix-16 butterfly costs more than it saves)
        stage_fixed<R, DIR, 16, 1, 128, 2>(b0, b1, rows, tw); sync_swap();
        stage_fixed<R, DIR, 8, 16, 128, 2>(b0, b1, rows, tw); sync_swap();
      } else {
        stage_fixed<R, DIR, 8, 1, 128, 2>(b0, b1, rows, tw); sync_swap();
        stage_fixed<R, DIR, 4, 8, 128, 2>(b0, b1, rows, tw); sync_swap();
        stage_fixed<R, DIR, 4, 32, 128, 2>(b0, b1, rows, tw); sync_swap();
      }
      return b0;
    case 64:
      stage_fixed<R, DIR, 8, 1, 64, 2>(b0, b1, rows, tw); sync_swap();
      stage_fixed<R, DIR, 8, 8, 64, 2>(b0, b1, rows, tw); sync_swap();
      return b0;
    case 32:
      stage_fixed<R, DIR, 8, 1, 32, 2>(b0, b1, rows, tw); sync_swap();
      stage_fixed<R, DIR, 4, 8, 32, 2>(b0, b1, rows, tw); sync_swap();
      return b0;
    case 16:
      stage_fixed<R, DIR, 4, 1, 16, 2>(b0, b1, rows, tw); sync_swap();
      stage_fixed<R, DIR, 4, 4, 16, 2>(b0, b1, rows, tw); sync_swap();
      return b0;
    case 24:
      stage_fixed<R, DIR, 8, 1, 24, 2>(b0, b1, rows, tw); sync_swap();
      stage_fixed<R, DIR, 3, 8, 24, 2>(b0, b1, rows, tw); sync_swap();
      return b0;
    case 12:
      stage_fixed<R, DIR, 4, 1, 12, 2>(b0, b1, rows, tw); sync_swap();
      stage_fixed<R, DIR, 3, 4, 12, 2>(b0, b1, rows, tw); sync_swap();
      return b0;
    case 8:
      stage_fixed<R, DIR, 8, 1, 8, 2>(b0, b1, rows, tw); sync_swap();
      return b0;
    default:
      return tile_fft<R, DIR, 8>(b0, b1, rows, p, tw);
  }
}

// The y / z column transforms (twiddle stride 1) of a tile of
// cols_per_tile(N) columns, 18 lines each, interleaved point by point: the
// common lengths with the host's plan (radix 16 where it saves a stage, radix
// 3 last) unrolled at compile time, others (one column per tile) through
// tile_fft.
template <class R, int DIR, int N>
__device__ __forceinline__ cpx<R>* fft_yz_fixed(cpx<R>* b0, cpx<R>* b1, const cpx<R>* tw) {
  constexpr int L = 18 * cols_per_tile(N);
  auto sync_swap = [&]() {
    __syncthreads();
    cpx<R>* t = b0;
    b0 = b1;
    b1 = t;
  };
  if constexpr (N == 256) {
    stage_fixed<R, DIR, 16, 1, 256, 1, L>(b0, b1, 1, tw); sync_swap();
    stage_fixed<R, DIR, 16, 16, 256, 1, L>(b0, b1, 1, tw); sync_swap();
  } else if constexpr (N == 128) {
    stage_fixed<R, DIR, 16, 1, 128, 1, L>(b0, b1, 1, tw); sync_swap();
    stage_fixed<R, DIR, 8, 16, 128, 1, L>(b0, b1, 1, tw); sync_swap();
  } else if constexpr (N == 64) {
    stage_fixed<R, DIR, 8, 1, 64, 1, L>(b0, b1, 1, tw); sync_swap();
    stage_fixed<R, DIR, 8, 8, 64, 1, L>(b0, b1, 1, tw); sync_swap();
  } else if constexpr (N == 48) {
    stage_fixed<R, DIR, 16, 1, 48, 1, L>(b0, b1, 1, tw); sync_swap();
    stage_fixed<R, DIR, 3, 16, 48, 1, L>(b0, b1, 1, tw); sync_swap();
  } else if constexpr (N == 32) {
    stage_fixed<R, DIR, 8, 1, 32, 1, L>(b0, b1, 1, tw); sync_swap();
    stage_fixed<R, DIR, 4, 8, 32, 1, L>(b0, b1, 1, tw); sync_swap();
  } else if constexpr (N == 24) {
    stage_fixed<R, DIR, 8, 1, 24, 1, L>(b0, b1, 1, tw); sync_swap();
    stage_fixed<R, DIR, 3, 8, 24, 1, L>(b0, b1, 1, tw); sync_swap();
  } else {
    static_assert(N == 16, "no compile-time plan for this length");
    stage_fixed<R, DIR, 16, 1, 16, 1, L>(b0, b1, 1, tw); sync_swap();
  }
  return b0;
}

// NF > 0: the compile-time plan of length NF (cols_per_tile(NF) columns per
// tile); otherwise the run-time plan p (one column per tile).
template <class R, int DIR, int NF>
__device__ cpx<R>* tile_fft_yz(cpx<R>* b0, cpx<R>* b1, const AxisPlan<R>& p, const cpx<R>* tw) {
  if constexpr (NF > 0) return fft_yz_fixed<R, DIR, NF>(b0, b1, tw);
  else return tile_fft<R, DIR, 16>(b0, b1, 1, p, tw);
}

}  // namespace mp
