// Green operator of the homogeneous micropolar reference medium, per
// wavevector (sm_103a).
//
// For a non-zero, non-Nyquist wavevector xi the strain / curvature
// fluctuations (e^, gamma^) produced by the polarizations (tau^, mu^) are
// those of the periodic displacement and micro-rotation amplitudes (u, phi)
// that balance t = A0 e + tau, m = B0 gamma + mu in Fourier space (the
// balance laws eq. momemtum_balance with the kinematics of eq. strains):
//
//   [(mu+kap) k^2 I + (lam+mu-kap) xi xi^T] u - 2 i kap (xi x phi) = f,
//   [(gam k^2 + 4 kap) I + (alp+bet) xi xi^T] phi - 2 i kap (xi x u) = g,
//   f_l = i xi_k tau^_kl,   g_l = i xi_k mu^_kl + eps_lkm tau^_km.
//
// Splitting along xi / across xi gives the closed form
//   u   = xi (xi.f) / ((lam + 2 mu) k^4) + [b P f - c (xi x g)] / D,
//   phi = xi (xi.g) / (((alp+bet+gam) k^2 + 4 kap) k^2) + [a P g - c (xi x f)] / D,
// a = (mu+kap) k^2, b = gam k^2 + 4 kap, c = -2 i kap, D = k^2 ((mu+kap) gam k^2 + 4 kap mu),
// P = I - xi xi^T / k^2; then e^_kl = i xi_k u_l + eps_lkm phi_m,
// gamma^_kl = i xi_l phi_k.  Lambda^1,2 of the paper act only at xi = 0,
// where the fluctuation is zero (the averages are prescribed).
#pragma once

#include "mp_common.cuh"

namespace mp {

// In-place: v[0..8] = tau^ -> e^, v[9..17] = mu^ -> gamma^, times `scale`.
// v may point to shared memory: every input is read before the first output
// is written, and only the 12 reals of f, g and of u, phi are kept in
// registers, never the 36 of the point itself.
template <class R>
__device__ __forceinline__ void green_point(const RefDev<R>& A0, R x1, R x2, R x3, cpx<R>* v,
                                            R scale) {
  const R xi[3] = {x1, x2, x3};
  // f = i xi . tau  (f_l = i xi_k tau_kl), g = i xi . mu + eps : tau
  cpx<R> f[3], g[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    cpx<R> a = cmake<R>(R(0), R(0)), b = cmake<R>(R(0), R(0));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      a = cadd(a, cscale(v[3 * k + l], xi[k]));
      b = cadd(b, cscale(v[9 + 3 * k + l], xi[k]));
    }
    f[l] = cmuli(a);
    g[l] = cmuli(b);
  }
  // (eps : tau)_1 = tau_23 - tau_32, _2 = tau_31 - tau_13, _3 = tau_12 - tau_21
  g[0] = cadd(g[0], csub(v[5], v[7]));
  g[1] = cadd(g[1], csub(v[6], v[2]));
  g[2] = cadd(g[2], csub(v[1], v[3]));

  const R k2 = x1 * x1 + x2 * x2 + x3 * x3;
  const R ik2 = R(1) / k2;
  const R a = (A0.mu + A0.kap) * k2;
  const R b = A0.gamma * k2 + R(4) * A0.kap;
  const R twok = R(2) * A0.kap;   // c = -i twok
  const R iD = R(1) / (k2 * ((A0.mu + A0.kap) * A0.gamma * k2 + R(4) * A0.kap * A0.mu));
  const R iL_u = ik2 * ik2 / (A0.lam + R(2) * A0.mu);
  const R iL_p = ik2 / ((A0.alpha + A0.beta + A0.gamma) * k2 + R(4) * A0.kap);

  cpx<R> xf = cmake<R>(R(0), R(0)), xg = cmake<R>(R(0), R(0));
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    xf = cadd(xf, cscale(f[l], xi[l]));
    xg = cadd(xg, cscale(g[l], xi[l]));
  }
  // cross products xi x g, xi x f
  cpx<R> cg[3], cf[3];
  cg[0] = csub(cscale(g[2], x2), cscale(g[1], x3));
  cg[1] = csub(cscale(g[0], x3), cscale(g[2], x1));
  cg[2] = csub(cscale(g[1], x1), cscale(g[0], x2));
  cf[0] = csub(cscale(f[2], x2), cscale(f[1], x3));
  cf[1] = csub(cscale(f[0], x3), cscale(f[2], x1));
  cf[2] = csub(cscale(f[1], x1), cscale(f[0], x2));

  cpx<R> u[3], ph[3];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    // P f = f - xi (xi.f)/k^2 ;  -c (xi x g) = i twok (xi x g)
    cpx<R> Pf = csub(f[l], cscale(xf, xi[l] * ik2));
    cpx<R> Pg = csub(g[l], cscale(xg, xi[l] * ik2));
    cpx<R> tu = cadd(cscale(Pf, b), cmuli(cscale(cg[l], twok)));
    cpx<R> tp = cadd(cscale(Pg, a), cmuli(cscale(cf[l], twok)));
    u[l] = cadd(cscale(xf, xi[l] * iL_u), cscale(tu, iD));
    ph[l] = cadd(cscale(xg, xi[l] * iL_p), cscale(tp, iD));
  }
  // e^_kl = i xi_k u_l + eps_lkm phi_m ; gamma^_kl = i phi_k xi_l, scaled, each
  // component written once.
  // eps_lkm phi_m: (1,2) -phi3, (2,1) +phi3, (1,3) +phi2, (3,1) -phi2, (2,3) -phi1, (3,2) +phi1
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    u[i] = cscale(u[i], scale);
    ph[i] = cscale(ph[i], scale);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int l = 0; l < 3; ++l) {
      cpx<R> ev = cmuli(cscale(u[l], xi[k]));
      if (k == 0 && l == 1) ev = csub(ev, ph[2]);
      if (k == 1 && l == 0) ev = cadd(ev, ph[2]);
      if (k == 0 && l == 2) ev = cadd(ev, ph[1]);
      if (k == 2 && l == 0) ev = csub(ev, ph[1]);
      if (k == 1 && l == 2) ev = csub(ev, ph[0]);
      if (k == 2 && l == 1) ev = cadd(ev, ph[0]);
      v[3 * k + l] = ev;
      v[9 + 3 * k + l] = cmuli(cscale(ph[k], xi[l]));
    }
  }
}

}  // namespace mp
