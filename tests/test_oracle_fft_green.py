"""Pins of the oracle's transforms and Green operator against the mathematics.

* Own FFT vs the brute-force triple sum and vs numpy.fft (P9).
* Green operator vs an independently derived closed form (block solve of the
  longitudinal / transverse parts), Hermitian symmetry, the projection
  property on compatible fields, the classical 1D limit, and the balance laws
  (eq. momemtum_balance) on its output (P6).
"""
import numpy as np
import pytest

from oracle import fft as offt
from oracle.constitutive import apply_A, apply_B, stiffness_A, stiffness_B
from oracle.green import (GreenOperator, assemble_operator, balance_residual, kinematics,
                          signed_frequencies, wavevectors)

RNG = np.random.default_rng(1234)


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 2, 2), (4, 2, 6), (3, 5, 4), (8, 4, 2)])
def test_fft_matches_bruteforce(shape):
    x = RNG.standard_normal(shape + (3,)) + 1j * RNG.standard_normal(shape + (3,))
    ref = offt.dft3_bruteforce(x)
    np.testing.assert_allclose(offt.fftn(x), ref, rtol=0, atol=1e-11 * np.abs(ref).max())
    np.testing.assert_allclose(offt.ifftn(ref), x, rtol=0, atol=1e-12 * np.abs(x).max())
    np.testing.assert_allclose(offt.dft3_bruteforce(ref, inverse=True), x, atol=1e-12)


@pytest.mark.parametrize("shape", [(16, 16, 16), (24, 12, 48), (6, 10, 14), (96, 2, 1)])
def test_fft_matches_library(shape):
    x = RNG.standard_normal(shape)
    ref = np.fft.fftn(x)
    got = offt.fftn(x)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    back = offt.ifftn(got)
    np.testing.assert_allclose(back.real, x, atol=1e-13)
    assert np.abs(back.imag).max() < 1e-13


def _reference():
    lam, mu, kap, al, be, ga = 20.0, 12.0, 3.0, 0.7, 1.1, 1.9
    return (lam, mu, kap, al, be, ga), stiffness_A(lam, mu, kap), stiffness_B(al, be, ga)


def _closed_form(xi, tau, mu_, mod):
    """Independent derivation: split the Fourier balance equations into the
    components along xi_hat and across it.  Along: (lambda+2mu) k^2 u_L = f_L and
    ((alpha+beta+gamma) k^2 + 4 kappa) phi_L = g_L.  Across: a u_T + c k x phi = f_T,
    b phi_T + c k x u = g_T with a = (mu+kappa) k^2, b = gamma k^2 + 4 kappa,
    c = -2 i kappa, whose determinant is D = k^2 ((mu+kappa) gamma k^2 + 4 kappa mu)."""
    lam, mu, kap, al, be, ga = mod
    f = 1j * np.einsum("k,kl->l", xi, tau)
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
    g = 1j * np.einsum("k,kl->l", xi, mu_) + np.einsum("lkm,km->l", eps, tau)
    k2 = xi @ xi
    kh = xi / np.sqrt(k2)
    PT = np.eye(3) - np.outer(kh, kh)
    a = (mu + kap) * k2
    b = ga * k2 + 4 * kap
    c = -2j * kap
    D = k2 * ((mu + kap) * ga * k2 + 4 * kap * mu)
    u = (kh @ f) * kh / ((lam + 2 * mu) * k2) + (b * PT @ f - c * np.cross(xi, g)) / D
    phi = (kh @ g) * kh / ((al + be + ga) * k2 + 4 * kap) + (a * PT @ g - c * np.cross(xi, f)) / D
    e = 1j * np.outer(xi, u) + np.einsum("lkm,m->kl", eps, phi)
    gam = 1j * np.outer(phi, xi)
    return e, gam


def test_green_matches_independent_closed_form():
    mod, A0, B0 = _reference()
    for _ in range(25):
        xi = RNG.standard_normal(3) * RNG.uniform(0.05, 5.0)
        tau = RNG.standard_normal((3, 3)) + 1j * RNG.standard_normal((3, 3))
        mu_ = RNG.standard_normal((3, 3)) + 1j * RNG.standard_normal((3, 3))
        op = GreenOperator(xi[None], np.ones(1, bool), A0, B0)
        e, g = op(tau[None], mu_[None])
        e_ref, g_ref = _closed_form(xi, tau, mu_, mod)
        scale = max(np.abs(e_ref).max(), np.abs(g_ref).max())
        assert np.abs(e[0] - e_ref).max() <= 1e-12 * scale
        assert np.abs(g[0] - g_ref).max() <= 1e-12 * scale


def test_operator_is_hermitian_and_balance_holds():
    mod, A0, B0 = _reference()
    xi = RNG.standard_normal((40, 3))
    K = assemble_operator(xi, A0, B0)
    # sign convention: K maps amplitudes to i xi . t, so -K is the (Hermitian) stiffness
    np.testing.assert_allclose(K, np.conj(np.swapaxes(K, 1, 2)), atol=1e-12)
    tau = RNG.standard_normal((40, 3, 3)) + 1j * RNG.standard_normal((40, 3, 3))
    mu_ = RNG.standard_normal((40, 3, 3)) + 1j * RNG.standard_normal((40, 3, 3))
    e, g = GreenOperator(xi, np.ones(40, bool), A0, B0)(tau, mu_)
    r1, r2 = balance_residual(xi, apply_A(A0, e) + tau, apply_B(B0, g) + mu_)
    assert np.abs(r1).max() < 1e-11 and np.abs(r2).max() < 1e-11


def test_projection_on_compatible_fields():
    """For compatible (e0, g0) = kinematics(u0, phi0), tau = -A0 e0 and
    mu = -B0 g0 are balanced by exactly (e0, g0)."""
    mod, A0, B0 = _reference()
    xi = RNG.standard_normal((30, 3))
    u0 = RNG.standard_normal((30, 3)) + 1j * RNG.standard_normal((30, 3))
    p0 = RNG.standard_normal((30, 3)) + 1j * RNG.standard_normal((30, 3))
    e0, g0 = kinematics(xi, u0, p0)
    e, g = GreenOperator(xi, np.ones(30, bool), A0, B0)(-apply_A(A0, e0), -apply_B(B0, g0))
    np.testing.assert_allclose(e, e0, atol=1e-12)
    np.testing.assert_allclose(g, g0, atol=1e-12)


def test_classical_uniaxial_limit():
    """A polarization tau_11 along xi = (k, 0, 0) gives e_11 = -tau_11 / (lambda + 2 mu)."""
    mod, A0, B0 = _reference()
    lam, mu = mod[0], mod[1]
    xi = np.array([[0.7, 0.0, 0.0]])
    tau = np.zeros((1, 3, 3), complex)
    tau[0, 0, 0] = 1.0 + 0.5j
    e, g = GreenOperator(xi, np.ones(1, bool), A0, B0)(tau, np.zeros_like(tau))
    assert abs(e[0, 0, 0] - (-(1.0 + 0.5j) / (lam + 2 * mu))) < 1e-14
    e_other = e[0].copy()
    e_other[0, 0] = 0
    assert np.abs(e_other).max() < 1e-14 and np.abs(g).max() < 1e-14


def test_wavevectors_and_masks():
    assert list(signed_frequencies(4)) == [0, 1, 2, -1]  # the Nyquist index is masked
    assert list(signed_frequencies(5)) == [0, 1, 2, -2, -1]
    xi, active = wavevectors((4, 6, 1), 0.5)
    # grid arrays are (N3, N2, N1) = (1, 6, 4)
    assert xi.shape == (1, 6, 4, 3)
    assert not active[0, 0, 0]
    assert not active[:, 3, :].any() and not active[:, :, 2].any()
    assert active.sum() == 1 * 5 * 3 - 1
    np.testing.assert_allclose(xi[0, 1, 1], [2 * np.pi / 2.0, 2 * np.pi / 3.0, 0.0])
    np.testing.assert_allclose(xi[0, 5, 3], [-2 * np.pi / 2.0, -2 * np.pi / 3.0, 0.0])
