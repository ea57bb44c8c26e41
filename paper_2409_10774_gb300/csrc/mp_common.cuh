// Shared device-side types of the micropolar FFT solver (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mp {

// ---------------------------------------------------------------- complex
template <class R>
struct cpx {
  R x, y;
};

template <class R>
__device__ __forceinline__ cpx<R> cmake(R a, R b) {
  cpx<R> c;
  c.x = a;
  c.y = b;
  return c;
}
template <class R>
__device__ __forceinline__ cpx<R> cadd(cpx<R> a, cpx<R> b) { return cmake<R>(a.x + b.x, a.y + b.y); }
template <class R>
__device__ __forceinline__ cpx<R> csub(cpx<R> a, cpx<R> b) { return cmake<R>(a.x - b.x, a.y - b.y); }
template <class R>
__device__ __forceinline__ cpx<R> cmul(cpx<R> a, cpx<R> b) {
  return cmake<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class R>
__device__ __forceinline__ cpx<R> cconj(cpx<R> a) { return cmake<R>(a.x, -a.y); }
template <class R>
__device__ __forceinline__ cpx<R> cscale(cpx<R> a, R s) { return cmake<R>(a.x * s, a.y * s); }
// multiply by i
template <class R>
__device__ __forceinline__ cpx<R> cmuli(cpx<R> a) { return cmake<R>(-a.y, a.x); }

// ---------------------------------------------------------------- phases
// Per-phase constants prepared on the host in FP64.  Moduli are kept in the
// field type R for the linear algebra; the scalar part of the radial return
// uses the double members.
template <class R>
struct PhaseDev {
  R lam, mu, kap, alpha, beta, gamma;   // eq. stiffnesses_iso
  R a1, a2, b1, b2;                     // eq. equiv_stress / equiv_couple_stress (b2 = 0 if gamma == beta)
  double tY, tH, mY, mH;                // eq. radius_1 / radius_2 (elastic: +inf yield)
  float tYf, tHf, mYf, mHf;             // the same rounded to single precision (FP32 fields)
  double ct, cm;                        // 2 a1 mu and b1 (gamma + beta) (eq. trial_stresses2)
  double inv_t, inv_m;                  // 1 / (tH + ct), 1 / (mH + cm)
  double ct_inv, tH_inv;                // ct / (tH + ct), tH / (tH + ct)
  double cm_inv, mH_inv;                // cm / (mH + cm), mH / (mH + cm)
  float inv_tf, inv_mf, ct_invf, tH_invf, cm_invf, mH_invf;  // the last six in single precision
  int elastic;
  int skew_m;                           // 1 when gamma > beta (b2 finite, skew part of m live)
  int ret32;                            // FP32 fields only: form the level return in FP32 too
};

// Reference medium (A0, B0) in the field type.
template <class R>
struct RefDev {
  R lam, mu, kap, alpha, beta, gamma;
};

// FFT plan of one axis: length N, radix sequence for the complex transform of
// length M (M = N / 2 for the packed real x-axis, M = N otherwise) and the
// device twiddle table W_T^k = exp(-2 pi i k / T), k < T, with T = N.
template <class R>
struct AxisPlan {
  int n;          // axis length
  int m;          // complex transform length
  int tstride;    // twiddle table stride: W_m^k = table[k * tstride]
  int nstages;
  int radix[10];
  const cpx<R>* tw;  // table of length n (n >= 1)
};

// Loop control of one cell over a window of batched rounds: Algorithm 2's
// convergence test (and the FP32 stagnation watch of the batched engine)
// taken on the device.  The error reduction of every round writes the cell's
// error row, counts the iteration and sets `stop` at the iteration where the
// host's test would end the cell's loop or change its schedule; the later
// rounds of the window skip a stopped cell.  The host then replays the rows
// through the same test.
struct RoundCtl {
  double tol, div_limit;
  double ref_err;    // stagnation watch (stall_step): error at the last new low
  double* rows;      // [max_rounds][8] the window's error rows
  int it;            // iterations of the current increment so far
  int target;        // prescribed iteration count of the increment, or -1
  int max_iter;
  int it_ref;        // iteration of the last significant new low (0: none yet)
  int stag_iters;    // iterations without a new low that stop the window (0: no watch)
  int adapt;         // 1: the window widens to twice the longest gap between lows (stall_step)
  int gap;           // longest gap between lows in the increment so far
  int max_rounds;    // rounds the window may run for this cell
  int rounds;        // rounds run (device-written)
  int stop;          // 1: no further round in this window (device-written)
};

// Per-cell device descriptor.
template <class R>
struct CellDev {
  int n1, n2, n3;
  int kx;                 // complex entries per spectral row: N1 / 2, or 1 when N1 == 1
  long long nvox;         // N1 N2 N3
  long long nspec;        // kx N2 N3
  double h;
  double inv_nvox;        // 1 / (N1 N2 N3)
  R two_pi_over_L[3];     // 2 pi / (N_j h)
  cpx<R>* spec;           // [nspec][18]  polarization / fluctuation spectra
  R* prev;                // [nvox][20]   e, gamma of the last iterate + scale factors f_t, f_m
  R* hist;                // [nvox][20]   h_t = t_n - A e_n (9), h_m = m_n - B gamma_n (9), phase id, 0
  double* pq;             // [nvox][2]    p_n, q_n
  R* elast;               // [nvox][18]   converged e, gamma of the step before (predictor)
  const uint16_t* phase;  // [nvox]
  const PhaseDev<R>* phases;
  RefDev<R> ref;
  AxisPlan<R> px, py, pz;
  R E[9], G[9];           // prescribed averages of the current step
  int* status;            // device status word: bit 0 = a bounded wait expired
  // batched (multi-cell) execution
  int rows_a;             // rows per pass-A work item
  long long items_a;      // pass-A work items
  double* ipart;          // [items_a][kErrPartials] per-item error partials
  double* apart;          // [ceil(nvox / 256)][kAvgPartials] per-chunk commit partials
  double* avg_out;        // row of this increment's homogenized averages
  double* err_out;        // [8] error of the last iteration (err, per field, status)
  int err_kind;           // eq. err metric: 0 = local (max), 1 = average
  // Increment form of the fixed-point iteration (pass A, iteration mode):
  // delta_in: the transformed field is e^{i+1} - e^i (else e^{i+1} - E);
  // delta_out: the polarization written is tau(e^i) - tau(e^{i-1}) (else tau - tau_c).
  int delta_in, delta_out;
  double* tmean;          // [kCellScalars]: <t>, <m> of the last iteration (18 constants subtracted
                          // before the transforms), then the loading-history magnitudes of the error
                          // measure: the largest ||<e>||, ||<t>||, ||<gamma>||, ||<m>|| of the
                          // converged increments so far
  int predict;            // commit: write the next increment's predictor
  double ratio;           // commit: (t_{n+1} - t_n) / (t_n - t_{n-1})
  // Manufactured source of the current increment ([nvox][18]: t^m - <t^m>,
  // m^m - <m^m>), subtracted from the polarization; NULL without a source.
  const R* src;
  // Batched rounds: the cell's loop control for the current window (NULL
  // outside a window; single-cell launches never set it).
  RoundCtl* rctl;
};

// Columns per tile of the y / z passes for a transform length n: short
// columns are grouped so that a tile holds about 256 points (the 288 threads
// of a block then have a butterfly or a Green-operator point each); lengths
// without a compile-time plan take one column per tile.
__host__ __device__ constexpr int cols_per_tile(int n) {
  return n == 16 ? 16 : n == 24 ? 10 : n == 32 ? 8 : n == 48 ? 5 : n == 64 ? 4 : n == 128 ? 2 : 1;
}
// Tiles of the y pass (columns (kz, kx), length N2) and of the z pass
// (columns (ky, kx), length N3) of a cell.
template <class R>
__host__ __device__ inline long long tiles_y(const CellDev<R>& c) {
  const long long cols = (long long)c.n3 * c.kx;
  const int cpt = cols_per_tile(c.n2);
  return (cols + cpt - 1) / cpt;
}
template <class R>
__host__ __device__ inline long long tiles_z(const CellDev<R>& c) {
  const long long cols = (long long)c.n2 * c.kx;
  const int cpt = cols_per_tile(c.n3);
  return (cols + cpt - 1) / cpt;
}

// The work of one multi-cell launch: entries e = 0..n_act-1 name cells
// (slots of `cells`); entry e owns global work items pre[e] .. pre[e+1]-1.
template <class R>
struct Work {
  const CellDev<R>* cells;
  const int* act;
  const long long* pre;
  int n_act;
};

// Stagnation watch of an FP32-mixed iteration (single cells and batches): a
// new low is an error below kStallDrop times the last low; kStallIters
// iterations without one end the full-form stage, kStallItersDelta the
// increment-form stage (the increment then finishes in FP64).
constexpr double kStallDrop = 0.99;
constexpr int kStallIters = 64;
constexpr int kStallItersDelta = 128;

// One step of the stagnation watch after iteration `it` with error `err`
// (above the tolerance), shared by the host and device loop tests: a new low
// (the first error, or one below kStallDrop times the last low) records its
// iteration and the longest gap between consecutive lows; returns true once
// no new low came for `window` iterations or, with adapt, for max(window,
// 2 x that longest gap): a slowly but steadily converging iteration keeps its
// pace between lows, while at a rounding floor the gaps grow without bound.
__host__ __device__ inline bool stall_step(double err, int it, int window, bool adapt, double& ref_err, int& it_ref,
                                           int& gap) {
  if (it_ref == 0 || err < kStallDrop * ref_err) {
    if (it_ref > 0 && it - it_ref > gap) gap = it - it_ref;
    ref_err = err;
    it_ref = it;
    return false;
  }
  const int w = (adapt && 2 * gap > window) ? 2 * gap : window;
  return it - it_ref >= w;
}

// Number of doubles in one block partial of the iteration error reduction:
// 4 maxima of |delta a|, 4 sums of |delta a|, 36 sums of e, t, gamma, m.
constexpr int kErrPartials = 44;
// Per-cell scalars kept on the device between launches (CellDev::tmean).
constexpr int kCellScalars = 22;
// Number of doubles in one block partial of the commit reduction:
// T (9), M (9), <e> (9), <gamma> (9), P, Q, T_eq, M_eq.
constexpr int kAvgPartials = 40;

}  // namespace mp
