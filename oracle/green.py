"""Green operator of the homogeneous micropolar reference medium (FP64).

Test infrastructure only (see the package docstring).

The paper uses Green tensors Gamma^1..4, Lambda^1,2 defined in its companion
work (Sec. 2.4, eq. micropolar_LippmannSchwinger_iteration), which is not
reproduced in the paper.  The oracle therefore writes the operator from its
definition: for every non-zero wavevector xi it finds the periodic
displacement and micro-rotation amplitudes (u^, phi^) whose strains (eq.
strains, in Fourier space e^_kl = i xi_k u^_l + eps_lkm phi^_m,
gamma^_kl = i xi_l phi^_k) make the generalized stresses
t^ = A0 e^ + tau^, m^ = B0 gamma^ + mu^ satisfy the balance laws without body
force or couple (eq. momemtum_balance):

    i xi_k t^_kl = 0,        i xi_k m^_kl + eps_lkm t^_km = 0.

The 6 x 6 linear map (u^, phi^) -> balance residual of (A0 e^, B0 gamma^) is
assembled column by column from those definitions and solved per wavevector.

Readings (where the paper is silent):
* Lambda^1,2 act on tau^0 = tau + A0 E, which differs from tau only at
  xi = 0; the xi = 0 fluctuation is zero so that <e> = E and <gamma> = Gamma
  exactly (prescribed averages, Sec. 2.4).  Hence tau^0 is never formed.
* Continuous frequencies xi_j = 2 pi n_j / (N_j h) with n_j in FFT order.
* Nyquist planes (even N_j, n_j = N_j / 2) get a zero fluctuation.
"""
from __future__ import annotations

import numpy as np

from .constitutive import EPS, apply_A, apply_B


def signed_frequencies(N):
    """Integer frequencies n_j in FFT order (0, 1, ..., -1)."""
    n = np.arange(N)
    return np.where(n <= N // 2, n, n - N)


def wavevectors(n, h):
    """Wavevector field xi[..., j] (j = direction x_{j+1}) on the (N3, N2, N1)
    grid, and a mask of the points that receive a non-zero fluctuation
    (xi != 0 and no Nyquist index)."""
    N1, N2, N3 = n
    f1, f2, f3 = signed_frequencies(N1), signed_frequencies(N2), signed_frequencies(N3)
    xi = np.zeros((N3, N2, N1, 3))
    xi[..., 0] = (2.0 * np.pi / (N1 * h)) * f1[None, None, :]
    xi[..., 1] = (2.0 * np.pi / (N2 * h)) * f2[:, None][None, :, :]
    xi[..., 2] = (2.0 * np.pi / (N3 * h)) * f3[:, None, None]
    active = np.ones((N3, N2, N1), dtype=bool)
    active[0, 0, 0] = False
    if N1 % 2 == 0:
        active[:, :, N1 // 2] = False
    if N2 % 2 == 0:
        active[:, N2 // 2, :] = False
    if N3 % 2 == 0:
        active[N3 // 2, :, :] = False
    return xi, active


def kinematics(xi, u, phi):
    """Fourier-space strains of eq. strains: e^_kl = i xi_k u^_l + eps_lkm phi^_m,
    gamma^_kl = i xi_l phi^_k."""
    e = 1j * xi[..., :, None] * u[..., None, :] + np.einsum("lkm,...m->...kl", EPS, phi)
    g = 1j * phi[..., :, None] * xi[..., None, :]
    return e, g


def balance_residual(xi, t, m):
    """Fourier-space balance laws of eq. momemtum_balance (no body force or
    couple): r1_l = i xi_k t^_kl, r2_l = i xi_k m^_kl + eps_lkm t^_km."""
    r1 = 1j * np.einsum("...k,...kl->...l", xi, t)
    r2 = 1j * np.einsum("...k,...kl->...l", xi, m) + np.einsum("lkm,...km->...l", EPS, t)
    return r1, r2


def assemble_operator(x, A0, B0):
    """K(xi): the 6 x 6 matrix mapping (u^, phi^) to the balance residual of
    (A0 e^, B0 gamma^), assembled column by column from eq. strains and eq.
    momemtum_balance.  x: (npts, 3) wavevectors."""
    npts = x.shape[0]
    K = np.zeros((npts, 6, 6), dtype=np.complex128)
    for c in range(6):
        u = np.zeros((npts, 3), dtype=np.complex128)
        phi = np.zeros((npts, 3), dtype=np.complex128)
        if c < 3:
            u[:, c] = 1.0
        else:
            phi[:, c - 3] = 1.0
        ek, gk = kinematics(x, u, phi)
        r1, r2 = balance_residual(x, apply_A(A0, ek), apply_B(B0, gk))
        K[:, :3, c] = r1
        K[:, 3:, c] = r2
    return K


class GreenOperator:
    """The reference medium's Green operator on one grid, with K(xi) assembled
    once (the paper notes the Green tensors may be precomputed, Sec. 2.4)."""

    def __init__(self, xi, active, A0, B0):
        self.xi = xi
        self.active = active
        self.x = xi[active]
        self.K = assemble_operator(self.x, A0, B0)

    def __call__(self, tau_hat, mu_hat):
        """Strain / curvature fluctuation spectra (e^, gamma^) produced by the
        polarization spectra (tau^, mu^): solve K (u^, phi^) = -residual(tau^, mu^)
        at every active wavevector, then apply the kinematics."""
        e_out = np.zeros(tau_hat.shape, dtype=np.complex128)
        g_out = np.zeros(mu_hat.shape, dtype=np.complex128)
        if self.x.shape[0] == 0:
            return e_out, g_out
        s1, s2 = balance_residual(self.x, tau_hat[self.active], mu_hat[self.active])
        rhs = -np.concatenate([s1, s2], axis=-1)
        sol = np.linalg.solve(self.K, rhs[..., None])[..., 0]
        ek, gk = kinematics(self.x, sol[:, :3], sol[:, 3:])
        e_out[self.active] = ek
        g_out[self.active] = gk
        return e_out, g_out


def green_apply(tau_hat, mu_hat, xi, active, A0, B0):
    """One-shot form of ``GreenOperator`` (tau_hat, mu_hat: complex (..., 3, 3);
    xi: (..., 3); active: bool (...))."""
    return GreenOperator(xi, active, A0, B0)(tau_hat, mu_hat)
