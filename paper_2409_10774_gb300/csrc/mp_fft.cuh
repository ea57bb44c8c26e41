// Shared-memory Stockham FFT building blocks (sm_103a).
//
// A tile holds `nlines` lines of a complex transform of length M in shared
// memory, line l at base + l * ls.  One stage of radix R (R in {2, 3, 4, 8})
// with Ns = product of the radices already applied reads butterfly j from
// in[j + r M / R] (r < R), multiplies input r by W_M^(r (j mod Ns) M / (Ns R)),
// takes the R-point DFT and writes output r to out[(j / Ns) Ns R + (j mod Ns)
// + r Ns].  After the last stage the line is in natural order (Stockham
// autosort; no bit reversal).  Transforms are unnormalised; the solver folds
// the 1 / (N1 N2 N3) of the inverse into the Green operator.
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

// One Stockham stage over all lines of a tile (all threads of the block).
template <class R, int DIR>
__device__ void stockham_stage(const cpx<R>* __restrict__ in, cpx<R>* __restrict__ out, int nlines,
                               int ls, int M, int radix, int Ns, const cpx<R>* __restrict__ tw,
                               int tstride) {
  const int nb = M / radix;
  const int total = nlines * nb;
  const int tstep = M / (Ns * radix);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int line = idx / nb;
    const int j = idx - line * nb;
    const int kk = j % Ns;
    const cpx<R>* src = in + line * ls;
    cpx<R> v[8];
    v[0] = src[j];
#pragma unroll
    for (int r = 1; r < 8; ++r) {
      if (r < radix) {
        cpx<R> x = src[j + r * nb];
        const int e = r * kk * tstep;  // < M
        v[r] = e == 0 ? x : cmul(x, twiddle<R, DIR>(tw, e * tstride));
      }
    }
    switch (radix) {
      case 2: dft2<R, DIR>(v); break;
      case 3: dft3<R, DIR>(v); break;
      case 4: dft4<R, DIR>(v); break;
      default: dft8<R, DIR>(v); break;
    }
    cpx<R>* dst = out + line * ls + (j / Ns) * Ns * radix + kk;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      if (r < radix) dst[r * Ns] = v[r];
    }
  }
}

// Full complex transform of every line of a tile; data starts in buf[0] and
// the result is returned (either buf[0] or buf[1]).  Ends with a barrier.
template <class R, int DIR>
__device__ cpx<R>* line_fft(cpx<R>* b0, cpx<R>* b1, int nlines, int ls, const AxisPlan<R>& p) {
  cpx<R>* in = b0;
  cpx<R>* out = b1;
  int Ns = 1;
  for (int s = 0; s < p.nstages; ++s) {
    stockham_stage<R, DIR>(in, out, nlines, ls, p.m, p.radix[s], Ns, p.tw, p.tstride);
    Ns *= p.radix[s];
    __syncthreads();
    cpx<R>* t = in;
    in = out;
    out = t;
  }
  return in;
}

}  // namespace mp
