// Transform plans of one axis (host side): the radix sequence and the twiddle
// table W_N^k = exp(-2 pi i k / N).  Header-only, with no dependency on the
// library context, so that every entry point (allocating or not) builds its
// plans from the same code; the compile-time stage sequences of the kernels
// (mp_fft.cuh, mp_kernels.cu) assume exactly these radix sequences.
#pragma once

#include <cmath>
#include <vector>

#include "mp_common.cuh"

namespace mp {

// Radix sequence of a complex transform of length m = 2^a 3^b.  Powers of two
// take as few stages as possible, radix 16 only where it saves one (allow16;
// the x axis, transformed inside pass A, is limited to radix 8); radix-3
// stages come last.
inline void radix_plan(int m, int* radix, int& nst, bool allow16) {
  nst = 0;
  int k2 = 0;
  while (m % 2 == 0) {
    m /= 2;
    ++k2;
  }
  int k3 = 0;
  while (m % 3 == 0) {
    m /= 3;
    ++k3;
  }
  static const int kPlan2[10][4] = {{0}, {2}, {4}, {8}, {16}, {8, 4}, {8, 8}, {16, 8}, {16, 16}, {8, 8, 8}};
  static const int kPlan2x[10][4] = {{0}, {2}, {4}, {8}, {4, 4}, {8, 4}, {8, 8}, {8, 4, 4}, {8, 8, 4}, {8, 8, 8}};
  static const int kLen2[10] = {0, 1, 1, 1, 1, 2, 2, 2, 2, 3};
  static const int kLen2x[10] = {0, 1, 1, 1, 2, 2, 2, 3, 3, 3};
  const int len = allow16 ? kLen2[k2] : kLen2x[k2];
  for (int i = 0; i < len; ++i) radix[nst++] = allow16 ? kPlan2[k2][i] : kPlan2x[k2][i];
  for (int i = 0; i < k3; ++i) radix[nst++] = 3;
}

// FFT plan of one axis and its twiddle table, computed in FP64 and rounded to
// R (host_tw receives n entries; p.tw is left for the caller to point at the
// device copy).  packed: the x axis, a real transform of length n through a
// complex one of length n / 2.
template <class R>
void axis_plan(int n, bool packed, AxisPlan<R>& p, cpx<R>* host_tw) {
  p.n = n;
  p.m = packed ? (n > 1 ? n / 2 : 1) : n;
  p.tstride = packed ? 2 : 1;
  radix_plan(p.m, p.radix, p.nstages, !packed);
  for (int k = 0; k < n; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)n;
    host_tw[k].x = (R)std::cos(a);
    host_tw[k].y = (R)(-std::sin(a));
  }
  p.tw = nullptr;
}

template <class R>
void axis_tables(int n, bool packed, AxisPlan<R>& p, std::vector<cpx<R>>& host_tw) {
  host_tw.resize(n);
  axis_plan<R>(n, packed, p, host_tw.data());
}

}  // namespace mp
