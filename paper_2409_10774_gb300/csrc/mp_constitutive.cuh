// Material-point update of the micropolar elastoplastic model (sm_103a).
//
// Implements Algorithm 1 (micropolar radial-return mapping) of Francis et al.
// with the closed-form plastic multipliers of eq. trial_stresses2.  Tensors
// are 9 values row-major (3k + l).  The trial stresses use the history form
// t_trial = h_t + A e with h_t = t_n - A e_n (eq. trial_stresses rearranged),
// and likewise m_trial = h_m + B gamma.
//
// Because Alg. 1 sets a2 = a1 mu / kappa and b2 = b1 (gamma + beta) /
// (gamma - beta), the symmetric and skew factors of each level coincide:
//   s_(kl) and s_[kl] are scaled by R1 / (R1 + 2 a1 mu (p - p_n)),
//   m_(kl) and m_[kl] are scaled by R2 / (R2 + b1 (gamma + beta) (q - q_n)),
// so the update is one scale factor per level.  When gamma == beta the skew
// part of m is identically zero and the b2 term of m_eq is dropped.
#pragma once

#include "mp_common.cuh"

namespace mp {

// 1 / sqrt(x) in FP64 for x > 0 by Newton's method on f(y) = 1/y^2 - x,
// y <- y (3 - x y^2) / 2, from the single-precision hardware estimate
// (relative error ~1e-7).  Two steps reach FP64 rounding.  Arguments outside
// the single-precision normal range take the FP64 library path.
// xf is x rounded to single precision (callers often have it at hand).
template <int STEPS>
__device__ __forceinline__ double rsqrt_newton(double x, float xf) {
  if (!(xf > 1e-36f && xf < 1e36f)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf(xf);
  const double hx = 0.5 * x;
#pragma unroll
  for (int i = 0; i < STEPS; ++i) y = y * fma(-hx * y, y, 1.5);
  return y;
}

// x >= 0 rounded toward zero to single precision (0 below the float normal
// range, FLT_MAX above it), with integer operations only.
__device__ __forceinline__ float float_rz(double x) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const int ex = (hi >> 20) & 0x7ff;
  if (hi <= 0 || ex < 1023 - 126) return 0.0f;
  if (ex > 1023 + 127) return 3.402823466e38f;
  return __int_as_float(((ex - 1023 + 127) << 23) | ((hi & 0xfffff) << 3) | (int)(lo >> 29));
}

// Closed-form return of one level in single precision (precision 2 only: FP32
// fields whose level return is FP32 as well).  The trial value q2 = (eq.
// stress)^2 is itself a single-precision quantity there, so the radius
// Y + H p_n, the multiplier increment and the scale factor are formed in
// single precision; only the accumulated multiplier p stays in FP64, so that
// small increments are not lost against it.  Returns false on the elastic
// branch.  The default FP32-field precision (1) forms all of these in FP64.
__device__ __forceinline__ bool return_level_f32(float q2, float Yf, float Hf, float inv, float c_inv, float H_inv,
                                                 double pn, double& p, float& f) {
  const float Rn = fmaf(Hf, float_rz(pn), Yf);
  if (q2 < Rn * Rn) return false;
  const float rinv = rsqrtf(q2);
  const float eq = q2 * rinv;
  p = pn + (double)((eq - Rn) * inv);
  f = fmaf(c_inv * Rn, rinv, H_inv);
  return true;
}

// t_kl = lam tr(e) d_kl + (mu + kappa) e_kl + (mu - kappa) e_lk  (eq. elast_constitutive_iso)
template <class R>
__device__ __forceinline__ void apply_A(R lam, R mu, R kap, const R* e, R* t) {
  const R tr = e[0] + e[4] + e[8];
  const R a = mu + kap, b = mu - kap;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int l = 0; l < 3; ++l) t[3 * k + l] = a * e[3 * k + l] + b * e[3 * l + k] + (k == l ? lam * tr : R(0));
  }
}

// m_kl = B_lkmn gamma_mn = alpha tr(gamma) d_kl + beta gamma_kl + gamma gamma_lk
template <class R>
__device__ __forceinline__ void apply_B(R al, R be, R ga, const R* g, R* m) {
  const R tr = g[0] + g[4] + g[8];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int l = 0; l < 3; ++l) m[3 * k + l] = be * g[3 * k + l] + ga * g[3 * l + k] + (k == l ? al * tr : R(0));
  }
}

// a1 |s_(kl)|^2 + a2 |s_[kl]|^2 of a deviator s (eq. equiv_stress squared)
template <class R>
__device__ __forceinline__ R eq_sq(const R* s, R c_sym, R c_skw, bool with_skw) {
  const R d = s[0] * s[0] + s[4] * s[4] + s[8] * s[8];
  const R y01 = R(0.5) * (s[1] + s[3]), k01 = R(0.5) * (s[1] - s[3]);
  const R y02 = R(0.5) * (s[2] + s[6]), k02 = R(0.5) * (s[2] - s[6]);
  const R y12 = R(0.5) * (s[5] + s[7]), k12 = R(0.5) * (s[5] - s[7]);
  R v = c_sym * (d + R(2) * (y01 * y01 + y02 * y02 + y12 * y12));
  if (with_skw) v += c_skw * R(2) * (k01 * k01 + k02 * k02 + k12 * k12);
  return v;
}

// Trial stress components (eq. trial_stresses, history form) with an explicit
// operation order, so that the same iterate always rebuilds bit-identical
// stresses wherever it is evaluated:
//   t_kl = h_kl + (mu + kappa) e_kl + (mu - kappa) e_lk [+ lam tr e],
//   m_kl = h_kl + beta gamma_kl + gamma gamma_lk [+ alpha tr gamma].
template <class R>
__device__ __forceinline__ R trial_t(const PhaseDev<R>& P, R h, R ei, R ej, bool diag, R tr) {
  R v = fma(P.mu - P.kap, ej, fma(P.mu + P.kap, ei, h));
  return diag ? fma(P.lam, tr, v) : v;
}
template <class R>
__device__ __forceinline__ R trial_m(const PhaseDev<R>& P, R h, R gi, R gj, bool diag, R tr) {
  R v = fma(P.gamma, gj, fma(P.beta, gi, h));
  return diag ? fma(P.alpha, tr, v) : v;
}

// Final stresses from the trial ones and the two scale factors:
// t = tr(t_trial)/3 d + f_t dev(t_trial), m = f_m m_trial.
template <class R>
__device__ __forceinline__ R vol_of(R t0, R t4, R t8) { return ((t0 + t4) + t8) * R(1.0 / 3.0); }
template <class R>
__device__ __forceinline__ R scaled_t(R ttr, bool diag, R vol, R ft) {
  return diag ? fma(ft, ttr - vol, vol) : ttr * ft;
}

// A level whose trial value q2 (FP32 fields) lies clearly inside the yield
// surface of radius Y + H p_n, judged in single precision with a margin well
// above its rounding, is elastic without the FP64 test; the other voxels take
// the FP64 test, whose outcome this screen never contradicts.  p_n is
// narrowed toward zero with integer operations (H >= 0, so the radius can
// only come out smaller: the screen stays on the safe side).
__device__ __forceinline__ bool surely_elastic_f32(float q2, float Yf, float Hf, double pn) {
  const float Rn = fmaf(Hf, float_rz(pn), Yf);
  return q2 < 0.999996f * (Rn * Rn);
}

// Algorithm 1, one level at a time: the macro level maps e (with the history
// ht, p_n) to t, p and the scale factor ft; the micro level maps gamma (hm,
// q_n) to m, q, fm.  The two levels share nothing but the phase, so a caller
// short of registers can run them one after the other.
// NEWTON: Newton steps of the FP64 reciprocal square root (2 reach FP64
// rounding; 1 leaves a relative error near 1e-14, ample for a scale factor
// that is rounded to FP32 fields, and is what the FP32-field iteration uses).
template <class R, int NEWTON = 2>
__device__ __forceinline__ void return_macro(const PhaseDev<R>& P, const R* e, const R* ht, double pn, R* t,
                                             double& p, R& ft) {
  const R tre = (e[0] + e[4]) + e[8];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int l = 0; l < 3; ++l) t[3 * k + l] = trial_t(P, ht[3 * k + l], e[3 * k + l], e[3 * l + k], k == l, tre);
  }
  p = pn;
  ft = R(1);
  const R vol = vol_of(t[0], t[4], t[8]);
  if (!P.elastic) {
    // eq. equiv_stress on the trial deviator
    R s[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) s[i] = t[i];
    s[0] -= vol; s[4] -= vol; s[8] -= vol;
    const R teq2r = eq_sq(s, P.a1, P.a2, true);
    float f32;
    if (sizeof(R) == 4 && P.ret32) {
      if (return_level_f32((float)teq2r, P.tYf, P.tHf, P.inv_tf, P.ct_invf, P.tH_invf, pn, p, f32)) ft = (R)f32;
    } else if (!(sizeof(R) == 4 && surely_elastic_f32((float)teq2r, P.tYf, P.tHf, pn))) {
      // the scalar solve in FP64 (for FP32 fields the trial value teq2r is
      // widened exactly)
      const double q2 = (double)teq2r;
      const double R1n = fma(P.tH, pn, P.tY);
      if (!(q2 < R1n * R1n)) {  // plastic: t_eq^trial >= t_Y + t_H p_n
        // eq. trial_stresses2: p - p_n = (t_eq^trial - R1(p_n)) / (t_H + 2 a1 mu).
        // Since R1(p) + 2 a1 mu (p - p_n) = t_eq^trial, the return factor
        // R1 / (R1 + 2 a1 mu (p - p_n)) = R1(p) / t_eq^trial
        //   = [2 a1 mu R1(p_n) + t_H t_eq^trial] / [(t_H + 2 a1 mu) t_eq^trial].
        const double rinv = rsqrt_newton<NEWTON>(q2, (float)teq2r);
        const double teq = q2 * rinv;
        p = pn + (teq - R1n) * P.inv_t;
        ft = (R)fma(P.ct_inv * R1n, rinv, P.tH_inv);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) t[i] = scaled_t(t[i], i % 4 == 0, vol, ft);
}

template <class R, int NEWTON = 2>
__device__ __forceinline__ void return_micro(const PhaseDev<R>& P, const R* g, const R* hm, double qn, R* m,
                                             double& q, R& fm) {
  const R trg = (g[0] + g[4]) + g[8];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int l = 0; l < 3; ++l) m[3 * k + l] = trial_m(P, hm[3 * k + l], g[3 * k + l], g[3 * l + k], k == l, trg);
  }
  q = qn;
  fm = R(1);
  if (!P.elastic) {
    // eq. equiv_couple_stress on the trial couple stress
    const R meq2r = eq_sq(m, P.b1, P.b2, P.skew_m != 0);
    float f32;
    if (sizeof(R) == 4 && P.ret32) {
      if (return_level_f32((float)meq2r, P.mYf, P.mHf, P.inv_mf, P.cm_invf, P.mH_invf, qn, q, f32)) fm = (R)f32;
    } else if (!(sizeof(R) == 4 && surely_elastic_f32((float)meq2r, P.mYf, P.mHf, qn))) {
      const double q2 = (double)meq2r;
      const double R2n = fma(P.mH, qn, P.mY);
      if (!(q2 < R2n * R2n)) {
        const double rinv = rsqrt_newton<NEWTON>(q2, (float)meq2r);
        const double meq = q2 * rinv;
        q = qn + (meq - R2n) * P.inv_m;
        fm = (R)fma(P.cm_inv * R2n, rinv, P.mH_inv);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) m[i] *= fm;
}

// Algorithm 1.  In: e, g (gamma), history ht, hm, p_n, q_n.  Out: t, m (final
// stresses), p, q and the scale factors ft, fm (1 on elastic branches).
template <class R>
__device__ __forceinline__ void radial_return(const PhaseDev<R>& P, const R* e, const R* g,
                                              const R* ht, const R* hm, double pn, double qn, R* t,
                                              R* m, double& p, double& q, R& ft, R& fm) {
  return_macro<R>(P, e, ht, pn, t, p, ft);
  return_micro<R>(P, g, hm, qn, m, q, fm);
}

// t_eq(t) and m_eq(m) of returned stresses (eq. equiv_stress and
// equiv_couple_stress), in the field type: for FP32 fields the stresses are
// themselves single-precision values, and their voxel averages are summed in
// FP64 (or compensated FP32) by the caller.
template <class R>
__device__ __forceinline__ void equivalents(const PhaseDev<R>& P, const R* t, const R* m, R& teq, R& meq) {
  const R vol = vol_of(t[0], t[4], t[8]);
  R s[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) s[i] = t[i];
  s[0] -= vol; s[4] -= vol; s[8] -= vol;
  teq = sqrt(eq_sq(s, P.a1, P.a2, true));
  meq = sqrt(eq_sq(m, P.b1, P.b2, P.skew_m != 0));
}

}  // namespace mp
