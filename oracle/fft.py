"""Discrete Fourier transforms for the oracle.

Test infrastructure only (see the package docstring).

The FFT-based scheme transforms the polarization fields and inverse-transforms
the strain / curvature fluctuations (Alg. 2, the Fourier-transform and inverse
steps of its while-loop; eq. micropolar_LippmannSchwinger_iteration).  The
transform convention is

    X[k] = sum_n x[n] exp(-2 pi i k n / N),   x[n] = (1/N) sum_k X[k] exp(+2 pi i k n / N)

applied along each of the three spatial axes.  Two independent evaluations are
provided:

* ``dft3_bruteforce`` - the triple sum written out (V x V phase matrix), for
  grids of at most a few hundred voxels;
* ``fftn`` / ``ifftn`` - a recursive decimation-in-time mixed-radix FFT
  (radix = smallest prime factor of the length, a direct DFT for larger prime
  factors), applied axis by axis.
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np

SPATIAL_AXES = (0, 1, 2)


def _smallest_factor(n: int) -> int:
    f = 2
    while f * f <= n:
        if n % f == 0:
            return f
        f += 1
    return n


@lru_cache(maxsize=None)
def _twiddles(n: int, r: int, sign: int) -> np.ndarray:
    """w[q, j, k] = exp(sign 2 pi i j (k + q m) / n), m = n / r."""
    m = n // r
    q = np.arange(r)[:, None, None]
    j = np.arange(r)[None, :, None]
    k = np.arange(m)[None, None, :]
    return np.exp(sign * 2j * np.pi * j * (k + q * m) / n)


@lru_cache(maxsize=None)
def _dft_matrix(n: int, sign: int) -> np.ndarray:
    k = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(k, k) / n)


def _fft_last_axis(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised DFT along the last axis with kernel exp(sign 2 pi i k n / N)."""
    n = x.shape[-1]
    if n == 1:
        return x.astype(np.complex128, copy=True)
    r = _smallest_factor(n)
    if r == n:
        # prime length: direct DFT
        return x @ _dft_matrix(n, sign).T
    m = n // r
    # decimation in time: sub-sequence j holds x[j], x[j + r], x[j + 2r], ...
    # and X[k + q m] = sum_j exp(sign 2 pi i j (k + q m) / n) S_j[k]
    subs = [_fft_last_axis(x[..., j::r], sign) for j in range(r)]
    w = _twiddles(n, r, sign)
    out = np.empty(x.shape[:-1] + (n,), dtype=np.complex128)
    for q in range(r):
        acc = w[q, 0] * subs[0]
        for j in range(1, r):
            acc = acc + w[q, j] * subs[j]
        out[..., q * m:(q + 1) * m] = acc
    return out


def fft_axis(x: np.ndarray, axis: int, inverse: bool = False) -> np.ndarray:
    """1D transform along ``axis`` (inverse includes the 1/N factor)."""
    y = np.moveaxis(np.asarray(x), axis, -1)
    out = _fft_last_axis(y, +1 if inverse else -1)
    if inverse:
        out = out / y.shape[-1]
    return np.moveaxis(out, -1, axis)


def fftn(x: np.ndarray, axes=SPATIAL_AXES) -> np.ndarray:
    """Forward 3D transform over ``axes`` (default: the three leading axes)."""
    out = np.asarray(x, dtype=np.complex128)
    for a in axes:
        out = fft_axis(out, a, inverse=False)
    return out


def ifftn(x: np.ndarray, axes=SPATIAL_AXES) -> np.ndarray:
    """Inverse 3D transform over ``axes`` (normalised by the voxel count)."""
    out = np.asarray(x, dtype=np.complex128)
    for a in axes:
        out = fft_axis(out, a, inverse=True)
    return out


def dft3_bruteforce(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Triple-sum 3D DFT over the three leading axes of ``x`` (any trailing
    component axes).  Cost O(V^2): meant for grids of up to ~8^3 voxels."""
    x = np.asarray(x, dtype=np.complex128)
    n3, n2, n1 = x.shape[:3]
    idx = np.stack(np.meshgrid(np.arange(n3), np.arange(n2), np.arange(n1), indexing="ij"),
                   axis=-1).reshape(-1, 3)
    sizes = np.array([n3, n2, n1], dtype=np.float64)
    phase = 2.0 * np.pi * ((idx[:, None, :] * idx[None, :, :]) / sizes).sum(axis=-1)
    sign = 1.0 if inverse else -1.0
    w = np.exp(sign * 1j * phase)
    flat = x.reshape(n3 * n2 * n1, -1)
    out = w @ flat
    if inverse:
        out = out / (n1 * n2 * n3)
    return out.reshape(x.shape)
