"""Pins of the oracle's material-point update (Algorithm 1).

* The stiffness tensors of eq. stiffnesses_iso reproduce the explicit
  symmetric / skew form of eq. elast_constitutive_iso.
* Radial-return invariants (P3): trace preserved, deviator (and the whole
  couple stress) scaled uniformly, returned stresses on the yield surfaces
  t_eq = t_Y + t_H p and m_eq = m_Y + m_H q, eq. trial_stresses2 satisfied,
  p >= p_n, elastic branch = identity.
* A simple-shear material point worked out by hand.
* Consistency with the continuum tangents of Appendix C (P4).
* The degenerate beta == gamma case (finite b2 limit) and elastic phases.
"""
import numpy as np
import pytest

import workloads as W
from oracle.constitutive import (apply_A, apply_B, deviator, m_eq, radial_return, skw,
                                 stiffness_A, stiffness_B, sym, t_eq, trace, a2_of, b2_of)
from oracle.tangent import tangent_A, tangent_B

PHASES = W.phase_record([
    # alpha = 0, gamma > beta
    {"lambda": 20.0, "mu": 12.0, "kappa": 3.0, "alpha": 0.0, "beta": 0.6, "gamma": 1.5,
     "tY": 0.05, "tH": 1.0, "mY": 0.04, "mH": 0.7, "a1": 1.5, "b1": 1.5},
    # alpha != 0, no hardening
    {"lambda": 8.0, "mu": 5.0, "kappa": 2.5, "alpha": 0.9, "beta": 0.2, "gamma": 2.0,
     "tY": 0.03, "tH": 0.0, "mY": 0.02, "mH": 0.0, "a1": 1.2, "b1": 0.8},
    # beta == gamma (degenerate b2)
    {"lambda": 20.0, "mu": 12.0, "kappa": 3.0, "alpha": 1.5, "beta": 1.5, "gamma": 1.5,
     "tY": 0.05, "tH": 1.0, "mY": 0.05, "mH": 1.0, "a1": 1.5, "b1": 1.5},
])


def _states(n, seed, ph):
    # magnitudes spread over a decade so that both branches occur at both levels
    s = W.random_material_states(n, seed, strain_scale=ph["tY"] / (2.0 * ph["mu"]),
                                 history_scale=0.5 * ph["tY"], p_scale=0.01)
    f = 10.0 ** np.random.default_rng(seed + 99).uniform(-1.2, 0.0, n)
    for k in ("e", "g", "e_n", "g_n", "t_n", "m_n"):
        s[k] = s[k] * f[:, None, None]
    if ph["gamma"] == ph["beta"]:
        s["m_n"] = sym(s["m_n"])  # admissible history: B maps to symmetric couple stress
    return s


def test_stiffness_tensors_match_explicit_isotropic_form():
    rng = np.random.default_rng(7)
    e = rng.standard_normal((5, 3, 3))
    g = rng.standard_normal((5, 3, 3))
    lam, mu, kap, al, be, ga = 2.0, 1.3, 0.4, 0.3, 0.7, 1.1
    t = apply_A(stiffness_A(lam, mu, kap), e)
    m = apply_B(stiffness_B(al, be, ga), g)
    I = np.eye(3)
    t_ref = lam * trace(e)[:, None, None] * I + 2 * mu * sym(e) + 2 * kap * skw(e)
    m_ref = al * trace(g)[:, None, None] * I + (be + ga) * sym(g) + (be - ga) * skw(g)
    np.testing.assert_allclose(t, t_ref, atol=1e-14)
    np.testing.assert_allclose(m, m_ref, atol=1e-14)
    # major symmetries stated with eq. elast_constitutive_aniso
    A = stiffness_A(lam, mu, kap)
    B = stiffness_B(al, be, ga)
    np.testing.assert_allclose(A, np.transpose(A, (2, 3, 0, 1)))   # A_klmn = A_mnkl
    np.testing.assert_allclose(B, np.transpose(B, (2, 3, 0, 1)))   # B_lkmn = B_mnlk


@pytest.mark.parametrize("pidx", [0, 1, 2])
def test_radial_return_invariants(pidx):
    ph = PHASES[pidx]
    s = _states(400, 11 + pidx, ph)
    t, m, p, q = radial_return(s["e"], s["g"], s["e_n"], s["g_n"], s["t_n"], s["m_n"],
                               s["p_n"], s["q_n"], ph)
    A = stiffness_A(ph["lambda"], ph["mu"], ph["kappa"])
    B = stiffness_B(ph["alpha"], ph["beta"], ph["gamma"])
    t_tr = s["t_n"] + apply_A(A, s["e"] - s["e_n"])
    m_tr = s["m_n"] + apply_B(B, s["g"] - s["g_n"])
    a1, a2, b1, b2 = ph["a1"], a2_of(ph), ph["b1"], b2_of(ph)
    teq_tr = t_eq(t_tr, a1, a2)
    meq_tr = m_eq(m_tr, b1, b2)
    R1n = ph["tY"] + ph["tH"] * s["p_n"]
    R2n = ph["mY"] + ph["mH"] * s["q_n"]
    macro = teq_tr >= R1n
    micro = meq_tr >= R2n
    assert 0.05 < macro.mean() < 0.97 and 0.05 < micro.mean() < 0.97
    # trace preserved, elastic branch identity
    np.testing.assert_allclose(trace(t), trace(t_tr), atol=1e-15)
    np.testing.assert_array_equal(t[~macro], t_tr[~macro])
    np.testing.assert_array_equal(p[~macro], s["p_n"][~macro])
    np.testing.assert_array_equal(m[~micro], m_tr[~micro])
    np.testing.assert_array_equal(q[~micro], s["q_n"][~micro])
    # deviator scaled uniformly by R1 / t_eq^trial; on the yield surface
    f = (ph["tY"] + ph["tH"] * p[macro]) / teq_tr[macro]
    np.testing.assert_allclose(deviator(t)[macro], f[:, None, None] * deviator(t_tr)[macro],
                               rtol=0, atol=1e-15)
    np.testing.assert_allclose(t_eq(t, a1, a2)[macro], ph["tY"] + ph["tH"] * p[macro], rtol=1e-13)
    # eq. trial_stresses2 and p >= p_n
    c = 2 * a1 * ph["mu"]
    np.testing.assert_allclose(p[macro], s["p_n"][macro] * c / (ph["tH"] + c)
                               + (teq_tr[macro] - ph["tY"]) / (ph["tH"] + c), rtol=1e-14)
    assert np.all(p >= s["p_n"]) and np.all(q >= s["q_n"])
    # micro level: whole couple stress scaled, on the yield surface for any alpha
    fm = (ph["mY"] + ph["mH"] * q[micro]) / meq_tr[micro]
    np.testing.assert_allclose(m[micro], fm[:, None, None] * m_tr[micro], rtol=0, atol=1e-15)
    np.testing.assert_allclose(m_eq(m, b1, b2)[micro], ph["mY"] + ph["mH"] * q[micro], rtol=1e-13)
    cm = b1 * (ph["gamma"] + ph["beta"])
    np.testing.assert_allclose(q[micro], s["q_n"][micro] * cm / (ph["mH"] + cm)
                               + (meq_tr[micro] - ph["mY"]) / (ph["mH"] + cm), rtol=1e-14)
    if b2 is None:
        assert np.abs(skw(m)).max() == 0.0


def test_simple_shear_by_hand():
    """e_12 = eps from a virgin state: t_12 = (mu+kappa) eps, t_21 = (mu-kappa) eps,
    t_eq^trial = eps sqrt(2 a1 mu (mu + kappa)); plastic return scales both."""
    ph = PHASES[0]
    mu, kap, a1, tY, tH = ph["mu"], ph["kappa"], ph["a1"], ph["tY"], ph["tH"]
    eps = 0.01
    e = np.zeros((1, 3, 3)); e[0, 0, 1] = eps
    z = np.zeros((1, 3, 3)); z0 = np.zeros(1)
    t, m, p, q = radial_return(e, z, z, z, z, z, z0, z0, ph)
    teq_tr = eps * np.sqrt(2 * a1 * mu * (mu + kap))
    p_ref = (teq_tr - tY) / (tH + 2 * a1 * mu)
    f = (tY + tH * p_ref) / teq_tr
    assert abs(p[0] - p_ref) < 1e-16
    assert abs(t[0, 0, 1] - f * (mu + kap) * eps) < 1e-15
    assert abs(t[0, 1, 0] - f * (mu - kap) * eps) < 1e-15
    mask = np.ones((3, 3), bool); mask[0, 1] = mask[1, 0] = False
    assert np.abs(t[0][mask]).max() == 0.0 and np.abs(m).max() == 0.0 and q[0] == 0.0


def test_elastic_phase_never_yields():
    row = {k: PHASES[0][k] for k in W.PHASE_FIELDS}
    row["elastic"] = 1
    ph = W.phase_record([row])[0]
    s = W.random_material_states(50, 5, strain_scale=1.0)
    t, m, p, q = radial_return(s["e"], s["g"], s["e_n"], s["g_n"], s["t_n"], s["m_n"],
                               s["p_n"], s["q_n"], ph)
    A = stiffness_A(ph["lambda"], ph["mu"], ph["kappa"])
    np.testing.assert_array_equal(t, s["t_n"] + apply_A(A, s["e"] - s["e_n"]))
    np.testing.assert_array_equal(p, s["p_n"])


@pytest.mark.parametrize("pidx", [0, 1])
def test_consistent_with_continuum_tangent(pidx):
    """From a state on both yield surfaces, a small increment along the loading
    path gives dt = A^ep de + O(de^2) and dm = B^ep dg + O(dg^2) (Appendix C,
    eq. continuum_tangent_A / _B, alpha = 0 as in Appendix B)."""
    ph = W.phase_record([{k: PHASES[pidx][k] for k in W.PHASE_FIELDS}])[0]
    ph["alpha"] = 0.0
    rng = np.random.default_rng(3 + pidx)
    e1 = 0.02 * rng.standard_normal((3, 3))
    g1 = 0.02 * rng.standard_normal((3, 3))
    z = np.zeros((3, 3))
    t1, m1, p1, q1 = radial_return(e1, g1, z, z, z, z, np.float64(0), np.float64(0), ph)
    assert p1 > 0 and q1 > 0
    At = tangent_A(t1, ph)
    Bt = tangent_B(m1, ph)
    # a non-proportional loading direction (proportional increments are exact)
    de0 = e1 + 0.5 * np.abs(e1).max() * rng.standard_normal((3, 3))
    dg0 = g1 + 0.5 * np.abs(g1).max() * rng.standard_normal((3, 3))
    errs = []
    for d in (1e-3, 1e-4, 1e-5):
        de, dg = d * de0, d * dg0
        t2, m2, _, _ = radial_return(e1 + de, g1 + dg, e1, g1, t1, m1, p1, q1, ph)
        et = np.abs((t2 - t1) - np.einsum("klmn,mn->kl", At, de)).max() / np.abs(t2 - t1).max()
        em = np.abs((m2 - m1) - np.einsum("lkmn,mn->kl", Bt, dg)).max() / np.abs(m2 - m1).max()
        errs.append(max(et, em))
    # first-order consistency: the relative mismatch shrinks linearly with the increment
    assert errs[0] > 1e-8, errs
    assert errs[1] < 0.2 * errs[0] and errs[2] < 0.2 * errs[1] and errs[2] < 1e-4, errs
