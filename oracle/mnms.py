"""Numerically manufactured solution MNMS-II of Appendix D.1 (FP64).

Test infrastructure only (see the package docstring).

Geometry: 4 x 4 x 4 voxels, unit cell L = 1 (h = 1/4); the centred 2 x 2 x 2
cube is the paper's phase 1 (table index 0), the surrounding layer its
phase 2 (table index 1); parameters as listed in Appendix D.1 (perfect
plasticity, alpha = 0).

Manufactured kinematics (eq. manufactured_displ_solutions, reading): the
periodic parts u*_i = phi*_i = t S(x), S = sin(2 pi x1) sin(2 pi x2) sin(2 pi x3),
produce the fluctuations, and the matrices of eq. manufactured_avg_strains are
taken as the prescribed averages, <e> = E^m(t), <gamma> = Gamma^m(t).  (The
printed linear terms E_ij x_j in u and Gamma_ij x_j in phi would give a
non-periodic skew strain eps_lkm Gamma_mj x_j; the prescribed-average reading
is the one compatible with the periodic scheme.)  Hence, from eq. strains,

    e^m_kl = E^m_kl + t (d_k S + eps_lkm S),     gamma^m_kl = Gamma^m_kl + t d_l S.

S sampled on 4 points per axis is band-limited (frequencies +-1 only), so the
Fourier derivative of the scheme reproduces d_k S exactly at the voxel centres.

Manufactured stresses: the continuum rate equations of Appendix C
(eq. stress_rates_with_continuum_tangent, p_dot_and_q_dot_EP) integrated in
time at every voxel, the paper's step (b).  The strain path is proportional
(e^m = t e1(x)), so the elastic stage is exact in closed form and the first
yield time of each level is t* = R / (equivalent stress of the unit-rate
elastic response); after t* the rates are integrated with classical RK4.
"""
from __future__ import annotations

import numpy as np

from workloads import phase_record

from .constitutive import (EPS, a2_of, apply_A, apply_B, b2_of, m_eq, stiffness_A, stiffness_B,
                           t_eq)
from .tangent import rates

E_RATE = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0], [7.0, 8.0, 9.0]])
G_RATE = np.array([[1.5, 2.5, 3.5], [4.5, 5.5, 6.5], [7.5, 8.5, 9.5]])

PHASES = phase_record([
    {"lambda": 1.0, "mu": 1.0, "kappa": 0.5, "alpha": 0.0, "beta": 0.5, "gamma": 1.0,
     "tY": 4.0, "tH": 0.0, "a1": 1.5, "mY": 4.0, "mH": 0.0, "b1": 1.5},
    {"lambda": 1.5, "mu": 1.5, "kappa": 0.75, "alpha": 0.0, "beta": 0.25, "gamma": 1.5,
     "tY": 4.5, "tH": 0.0, "a1": 1.5, "mY": 4.5, "mH": 0.0, "b1": 1.5},
])


def phase_map():
    pm = np.ones((4, 4, 4), dtype=np.uint16)
    pm[1:3, 1:3, 1:3] = 0
    return pm


def unit_rate_fields(N=4, L=1.0):
    """(e1, g1) with e^m = t e1, gamma^m = t g1 at the voxel centres."""
    h = L / N
    x = (np.arange(N) + 0.5) * h
    k = 2.0 * np.pi / L
    s1, c1 = np.sin(k * x), np.cos(k * x)
    # arrays indexed [x3][x2][x1]
    S = s1[:, None, None] * s1[None, :, None] * s1[None, None, :]
    dS = np.zeros((N, N, N, 3))
    dS[..., 0] = k * s1[:, None, None] * s1[None, :, None] * c1[None, None, :]
    dS[..., 1] = k * s1[:, None, None] * c1[None, :, None] * s1[None, None, :]
    dS[..., 2] = k * c1[:, None, None] * s1[None, :, None] * s1[None, None, :]
    ones = np.ones(3)
    # e_kl = d_k u_l + eps_lkm phi_m with u_l = phi_m = S
    e1 = E_RATE + dS[..., :, None] * ones[None, :] + S[..., None, None] * np.einsum("lkm,m->kl", EPS, ones)
    # gamma_kl = d_l phi_k
    g1 = G_RATE + ones[:, None] * dS[..., None, :]
    return e1, g1


def problem(n_steps=100, tol=1e-9):
    time = np.linspace(0.0, 1.0, n_steps + 1)
    return dict(n=(4, 4, 4), h=0.25, phase=phase_map(), phases=PHASES, time=time,
                E=time[:, None, None] * E_RATE[None], G=time[:, None, None] * G_RATE[None],
                tol=tol, err_kind="local", ref_kind="mean", ref_moduli=None, max_iter=100000,
                name="mnms-4^3")


def manufactured_stresses(times, substeps=4):
    """t^m(x, t), m^m(x, t) at the requested times (ascending, starting at 0).

    Returns arrays of shape (len(times), 4, 4, 4, 3, 3)."""
    e1, g1 = unit_rate_fields()
    pm = phase_map()
    nt = len(times)
    tm = np.zeros((nt, 4, 4, 4, 3, 3))
    mm = np.zeros((nt, 4, 4, 4, 3, 3))
    for idx in np.ndindex(4, 4, 4):
        ph = PHASES[int(pm[idx])]
        A = stiffness_A(ph["lambda"], ph["mu"], ph["kappa"])
        B = stiffness_B(ph["alpha"], ph["beta"], ph["gamma"])
        ed, gd = e1[idx], g1[idx]
        # elastic responses to the unit-rate path and first-yield times
        t_unit = apply_A(A, ed)
        m_unit = apply_B(B, gd)
        ty = ph["tY"] / t_eq(t_unit, ph["a1"], a2_of(ph))
        my = ph["mY"] / m_eq(m_unit, ph["b1"], b2_of(ph))
        t_state = np.zeros((3, 3))
        m_state = np.zeros((3, 3))
        clock = 0.0
        for j, target in enumerate(times):
            while clock < target - 1e-15:
                # advance to the next event (yield time) or the target
                nxt = target
                for ev in (ty, my):
                    if clock < ev < nxt:
                        nxt = ev
                macro = clock >= ty
                micro = clock >= my
                if not macro and not micro:
                    # purely elastic stage: exact
                    t_state = nxt * t_unit
                    m_state = nxt * m_unit
                else:
                    dt = (nxt - clock) / substeps
                    for _ in range(substeps):
                        def f(ts, ms):
                            td, md, _, _ = rates(ts, ms, ed, gd, ph, macro, micro, A, B)
                            return td, md
                        k1 = f(t_state, m_state)
                        k2 = f(t_state + 0.5 * dt * k1[0], m_state + 0.5 * dt * k1[1])
                        k3 = f(t_state + 0.5 * dt * k2[0], m_state + 0.5 * dt * k2[1])
                        k4 = f(t_state + dt * k3[0], m_state + dt * k3[1])
                        t_state = t_state + dt / 6.0 * (k1[0] + 2 * k2[0] + 2 * k3[0] + k4[0])
                        m_state = m_state + dt / 6.0 * (k1[1] + 2 * k2[1] + 2 * k3[1] + k4[1])
                    if not macro:
                        t_state = nxt * t_unit
                    if not micro:
                        m_state = nxt * m_unit
                clock = nxt
            tm[(j,) + idx] = t_state
            mm[(j,) + idx] = m_state
    return tm, mm
