"""Continuum elastoplastic tangents and rate equations (Appendix C), FP64.

Test infrastructure only (see the package docstring).

Used to pin the radial return (its consistency with the continuum tangent for
small increments) and to integrate the manufactured stresses of Appendix D.1
independently of Algorithm 1.

Index conventions follow the paper: A[k, l, m, n] = A_klmn and
B[l, k, m, n] = B_lkmn with slots in the written order (see
``constitutive.stiffness_B``); N = df/dt (eq. dfdt) and g = dg/dm (eq. dgdm),
with the micro-plastic flow gamma^p_dot_lk = lambda_2 dg/dm_kl (eq.
plastic_flow_intext).
"""
from __future__ import annotations

import numpy as np

from .constitutive import (a2_of, b2_of, deviator, m_eq, skw, stiffness_A, stiffness_B, sym,
                           t_eq)


def df_dt(t, a1, a2):
    """eq. dfdt: (a1 s_(kl) + a2 s_[kl]) / t_eq(t)."""
    s = deviator(t)
    return (a1 * sym(s) + a2 * skw(s)) / t_eq(t, a1, a2)[..., None, None]


def dg_dm(m, b1, b2):
    """eq. dgdm: (b1 m_(kl) + b2 m_[kl]) / m_eq(m) (b2 None -> skew term absent)."""
    val = b1 * sym(m)
    if b2 is not None:
        val = val + b2 * skw(m)
    return val / m_eq(m, b1, b2)[..., None, None]


def tangent_A(t, ph):
    """Plastic branch of eq. continuum_tangent_A (df/dp = -t_H):
    A_klmn - A_klrs N_rs N_pq A_pqmn / (N_ab A_abcd N_cd + t_H)."""
    A = stiffness_A(ph["lambda"], ph["mu"], ph["kappa"])
    N = df_dt(t, ph["a1"], a2_of(ph))
    AN = np.einsum("klrs,rs->kl", A, N)
    NA = np.einsum("pq,pqmn->mn", N, A)
    den = np.einsum("ab,abcd,cd->", N, A, N) + ph["tH"]
    return A - np.einsum("kl,mn->klmn", AN, NA) / den


def tangent_B(m, ph):
    """Plastic branch of eq. continuum_tangent_B (dg/dq = -m_H), slots (l,k,m,n):
    B_lkmn - B_lkrs g_sr g_pq B_qpmn / (g_ba B_abcd g_dc + m_H)."""
    B = stiffness_B(ph["alpha"], ph["beta"], ph["gamma"])
    g = dg_dm(m, ph["b1"], b2_of(ph))
    Bg = np.einsum("lkrs,sr->lk", B, g)
    gB = np.einsum("pq,qpmn->mn", g, B)
    den = np.einsum("ba,abcd,dc->", g, B, g) + ph["mH"]
    return B - np.einsum("lk,mn->lkmn", Bg, gB) / den


def rates(t, m, e_dot, g_dot, ph, macro_plastic, micro_plastic, A=None, B=None):
    """Stress-rate equations with the loading conditions of eq.
    p_dot_and_q_dot_EP, for material points whose macro / micro level is on
    its yield surface (boolean flags).  Returns (t_dot, m_dot, p_dot, q_dot)
    for single 3x3 tensors.  A, B: the phase's stiffness tensors (built from
    ``ph`` when not given)."""
    if A is None:
        A = stiffness_A(ph["lambda"], ph["mu"], ph["kappa"])
    if B is None:
        B = stiffness_B(ph["alpha"], ph["beta"], ph["gamma"])
    p_dot = 0.0
    q_dot = 0.0
    if macro_plastic:
        N = df_dt(t, ph["a1"], a2_of(ph))
        num = np.einsum("kl,klmn,mn->", N, A, e_dot)
        den = np.einsum("ab,abcd,cd->", N, A, N) + ph["tH"]
        p_dot = max(num, 0.0) / den
        t_dot = np.einsum("klmn,mn->kl", A, e_dot - p_dot * N)
    else:
        t_dot = np.einsum("klmn,mn->kl", A, e_dot)
    if micro_plastic:
        g = dg_dm(m, ph["b1"], b2_of(ph))
        num = np.einsum("kl,lkmn,mn->", g, B, g_dot)
        den = np.einsum("ba,abcd,dc->", g, B, g) + ph["mH"]
        q_dot = max(num, 0.0) / den
        # gamma^p_dot_mn = q_dot dg/dm_nm
        m_dot = np.einsum("lkmn,mn->kl", B, g_dot - q_dot * g.T)
    else:
        m_dot = np.einsum("lkmn,mn->kl", B, g_dot)
    return t_dot, m_dot, p_dot, q_dot
