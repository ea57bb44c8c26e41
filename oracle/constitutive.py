"""Isotropic micropolar elastoplasticity at a material point (FP64).

Test infrastructure only (see the package docstring).

Tensor arrays carry their two indices last: ``e[..., k, l]`` is e_kl.

Follows the paper's Sec. 2.2-2.3:
* stiffness tensors A_klmn, B_lkmn of eq. stiffnesses_iso, applied as
  t_kl = A_klmn e_mn and m_kl = B_lkmn gamma_mn (eq. elast_constitutive_aniso);
* equivalent stress t_eq (eq. equiv_stress) on the deviator s (defined right
  after it) and equivalent couple stress m_eq (eq. equiv_couple_stress);
* Algorithm 1 (micropolar radial-return mapping) with the closed-form p, q of
  eq. trial_stresses2 (derived in Appendix B).

Readings where the paper is silent or degenerate:
* b2 = b1 (gamma + beta) / (gamma - beta) (Alg. 1) is infinite when
  gamma == beta.  Then m_[kl] is identically zero (B maps every curvature to a
  symmetric couple stress and the history starts at zero), so the b2 term of
  m_eq is dropped and the skew scale factor uses its finite limit
  b2 (gamma - beta) = b1 (gamma + beta).
* An ``elastic`` phase has infinite yield stresses: both levels always take
  the elastic branch.
* alpha != 0 is handled exactly as Alg. 1 states (one scale factor per
  symmetric / skew part of m), although Appendix B derives it for alpha = 0.
"""
from __future__ import annotations

import numpy as np

I3 = np.eye(3)

# Levi-Civita symbol eps[i, j, k]
EPS = np.zeros((3, 3, 3))
EPS[0, 1, 2] = EPS[1, 2, 0] = EPS[2, 0, 1] = 1.0
EPS[0, 2, 1] = EPS[2, 1, 0] = EPS[1, 0, 2] = -1.0


def stiffness_A(lam, mu, kappa):
    """A_klmn = lam d_kl d_mn + (mu + kappa) d_km d_ln + (mu - kappa) d_kn d_lm,
    stored as A[k, l, m, n] (eq. stiffnesses_iso)."""
    d = I3
    return (lam * np.einsum("kl,mn->klmn", d, d)
            + (mu + kappa) * np.einsum("km,ln->klmn", d, d)
            + (mu - kappa) * np.einsum("kn,lm->klmn", d, d))


def stiffness_B(alpha, beta, gamma):
    """B_lkmn = alpha d_kl d_mn + beta d_km d_ln + gamma d_kn d_lm, stored with
    its index slots in the order written, B[l, k, m, n] (eq. stiffnesses_iso)."""
    d = I3
    return (alpha * np.einsum("kl,mn->lkmn", d, d)
            + beta * np.einsum("km,ln->lkmn", d, d)
            + gamma * np.einsum("kn,lm->lkmn", d, d))


def apply_A(A, e):
    """t_kl = A_klmn e_mn."""
    return np.einsum("klmn,...mn->...kl", A, e)


def apply_B(B, g):
    """m_kl = B_lkmn gamma_mn (note the swapped first pair, eq. elast_constitutive_aniso)."""
    return np.einsum("lkmn,...mn->...kl", B, g)


def transpose(V):
    return np.swapaxes(V, -1, -2)


def sym(V):
    """V_(kl) (eq. sym_and_skew)."""
    return 0.5 * (V + transpose(V))


def skw(V):
    """V_[kl] (eq. sym_and_skew)."""
    return 0.5 * (V - transpose(V))


def trace(V):
    return np.trace(V, axis1=-2, axis2=-1)


def deviator(t):
    """s_kl = t_kl - t_nn d_kl / 3."""
    return t - trace(t)[..., None, None] * I3 / 3.0


def frob2(V):
    return np.einsum("...kl,...kl->...", V, V)


def a2_of(ph):
    """a2 = a1 mu / kappa (Alg. 1, eq. equivalent_trial_stress_assumption)."""
    return ph["a1"] * ph["mu"] / ph["kappa"]


def b2_of(ph):
    """b2 = b1 (gamma + beta) / (gamma - beta), or None when gamma == beta
    (the skew part of m is then identically zero)."""
    if ph["gamma"] == ph["beta"]:
        return None
    return ph["b1"] * (ph["gamma"] + ph["beta"]) / (ph["gamma"] - ph["beta"])


def t_eq(t, a1, a2):
    """Equivalent stress of eq. equiv_stress."""
    s = deviator(t)
    return np.sqrt(a1 * frob2(sym(s)) + a2 * frob2(skw(s)))


def m_eq(m, b1, b2):
    """Equivalent couple stress of eq. equiv_couple_stress (b2 None -> skew term
    dropped, see the module docstring)."""
    val = b1 * frob2(sym(m))
    if b2 is not None:
        val = val + b2 * frob2(skw(m))
    return np.sqrt(val)


def radial_return(e, g, e_n, g_n, t_n, m_n, p_n, q_n, ph):
    """Algorithm 1 for one phase ``ph`` (a mapping of scalar parameters) over a
    batch of material points.  Tensors (..., 3, 3), p_n and q_n shape (...).

    Returns (t, m, p, q)."""
    A = stiffness_A(ph["lambda"], ph["mu"], ph["kappa"])
    B = stiffness_B(ph["alpha"], ph["beta"], ph["gamma"])
    a1, b1 = ph["a1"], ph["b1"]
    mu, kappa, beta, gamma = ph["mu"], ph["kappa"], ph["beta"], ph["gamma"]

    # trial stresses, eq. trial_stresses
    t_tr = t_n + apply_A(A, e - e_n)
    m_tr = m_n + apply_B(B, g - g_n)
    # a2, b2 (Alg. 1)
    a2 = a2_of(ph)
    b2 = b2_of(ph)
    teq_tr = t_eq(t_tr, a1, a2)
    meq_tr = m_eq(m_tr, b1, b2)

    t = t_tr.copy()
    m = m_tr.copy()
    p = np.array(p_n, dtype=np.float64, copy=True)
    q = np.array(q_n, dtype=np.float64, copy=True)
    if ph["elastic"]:
        return t, m, p, q

    # macro level
    tY, tH = ph["tY"], ph["tH"]
    plastic = ~(teq_tr < tY + tH * p_n)
    if np.any(plastic):
        c = 2.0 * a1 * mu
        pn = np.asarray(p_n)[plastic]
        p_new = pn * c / (tH + c) + (teq_tr[plastic] - tY) / (tH + c)       # eq. trial_stresses2
        R1 = tY + tH * p_new
        f_sym = R1 / (R1 + 2.0 * (p_new - pn) * a1 * mu)
        f_skw = R1 / (R1 + 2.0 * (p_new - pn) * a2 * kappa)
        s_tr = deviator(t_tr[plastic])
        t[plastic] = (trace(t_tr[plastic])[..., None, None] * I3 / 3.0
                      + f_sym[..., None, None] * sym(s_tr) + f_skw[..., None, None] * skw(s_tr))
        p[plastic] = p_new

    # micro level
    mY, mH = ph["mY"], ph["mH"]
    plastic = ~(meq_tr < mY + mH * q_n)
    if np.any(plastic):
        c = b1 * (gamma + beta)
        # b2 (gamma - beta); its finite limit when gamma == beta
        c_skw = c if b2 is None else b2 * (gamma - beta)
        qn = np.asarray(q_n)[plastic]
        q_new = qn * c / (mH + c) + (meq_tr[plastic] - mY) / (mH + c)       # eq. trial_stresses2
        R2 = mY + mH * q_new
        f_sym = R2 / (R2 + (q_new - qn) * c)
        f_skw = R2 / (R2 + (q_new - qn) * c_skw)
        mt = m_tr[plastic]
        m[plastic] = f_sym[..., None, None] * sym(mt) + f_skw[..., None, None] * skw(mt)
        q[plastic] = q_new
    return t, m, p, q


def phase_moduli_fields(phase_map, phases):
    """Per-voxel stiffness application helpers: returns a list of
    (mask, A_tensor, B_tensor, row) for each phase present."""
    out = []
    for idx in np.unique(phase_map):
        row = phases[int(idx)]
        out.append((phase_map == idx,
                    stiffness_A(row["lambda"], row["mu"], row["kappa"]),
                    stiffness_B(row["alpha"], row["beta"], row["gamma"]), row))
    return out


def radial_return_field(e, g, e_n, g_n, t_n, m_n, p_n, q_n, phase_map, phases):
    """Algorithm 1 applied voxel by voxel over a heterogeneous field."""
    t = np.empty_like(e)
    m = np.empty_like(g)
    p = np.empty_like(p_n)
    q = np.empty_like(q_n)
    for idx in np.unique(phase_map):
        mask = phase_map == idx
        ph = phases[int(idx)]
        t[mask], m[mask], p[mask], q[mask] = radial_return(
            e[mask], g[mask], e_n[mask], g_n[mask], t_n[mask], m_n[mask], p_n[mask], q_n[mask], ph)
    return t, m, p, q


def equivalent_fields(t, m, phase_map, phases):
    """Per-voxel t_eq(t), m_eq(m) with each voxel's own a1, a2, b1, b2."""
    teq = np.empty(t.shape[:-2])
    meq = np.empty(m.shape[:-2])
    for idx in np.unique(phase_map):
        mask = phase_map == idx
        ph = phases[int(idx)]
        teq[mask] = t_eq(t[mask], ph["a1"], a2_of(ph))
        meq[mask] = m_eq(m[mask], ph["b1"], b2_of(ph))
    return teq, meq
