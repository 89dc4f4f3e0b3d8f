"""The oracle's own discrete Fourier transform (TEST INFRASTRUCTURE ONLY).

A plain recursive Cooley-Tukey FFT for any length, in FP64 numpy, written from the
definition of the DFT:

    X[k] = sum_{j=0}^{n-1} x[j] exp(sign 2 pi i j k / n),   sign = -1 forward, +1 inverse,

unnormalised in both directions (the 1/n of the inverse transform is applied by the caller,
as Section 2.1's convention puts it on the inverse).

Splitting n = p m with the input index j = j1 + p j2 (j1 < p, j2 < m) and the output index
k = k2 + m k1 (k2 < m, k1 < p) gives

    X[k2 + m k1] = sum_{j1} exp(sign 2 pi i j1 k1 / p) [exp(sign 2 pi i j1 k2 / n) Y_j1[k2]],
    Y_j1[k2]     = sum_{j2} x[j1 + p j2] exp(sign 2 pi i j2 k2 / m),

that is: p transforms of length m of the interleaved subsequences (the recursion), a
twiddle factor, and one p-point DFT per output column evaluated as a dense p x p matrix
product.  p is the largest divisor of n up to 16 (16, 12, 8, 6, 4, 3, 2); lengths up to 16,
and a length with no such divisor, are transformed by the definition (an n x n matrix
product).  Every step is the
definition above; nothing is blocked or reordered beyond it.

Real transforms over the last three axes follow numpy's conventions (the half spectrum of a
real DFT along the last axis; the inverse reads only the real parts of the zero and Nyquist
bins of that axis) so that the spectral layout of the rest of the oracle is unchanged.
"""
from __future__ import annotations

import numpy as np

_RADICES = (16, 12, 8, 6, 4, 3, 2)


def dft_matrix(n: int, sign: int) -> np.ndarray:
    """F[k, j] = exp(sign 2 pi i j k / n); the exponent j k is reduced mod n exactly."""
    jk = np.outer(np.arange(n), np.arange(n)) % n
    return np.exp(sign * 2j * np.pi * jk / n)


def _fft_mid(x: np.ndarray, sign: int) -> np.ndarray:
    """Unnormalised DFT along the middle axis of a contiguous complex array of shape
    (A, n, R): every (a, r) column is transformed independently."""
    A, n, R = x.shape
    p = next((r for r in _RADICES if n % r == 0 and r < n), None) if n > 16 else None
    if p is None:
        # up to 16 points, or a length without a small divisor: the definition itself,
        # X[a, k, r] = sum_j F[k, j] x[a, j, r] with the n x n DFT matrix (for R = 1 the
        # same product written as X[a, :] = x[a, :] F^T)
        if R == 1:
            return np.matmul(x.reshape(A, n), dft_matrix(n, sign).T).reshape(A, n, 1)
        return np.matmul(dft_matrix(n, sign), x)
    m = n // p
    # j = j1 + p j2: viewed as (A, m, p R), the subsequence j1 sits in the trailing axis, so
    # one transform of length m over the middle axis gives Y[a, k2, j1, r] for every j1
    y = _fft_mid(x.reshape(A, m, p * R), sign).reshape(A, m, p, R)
    j1 = np.arange(p)[None, None, :, None]
    k2 = np.arange(m)[None, :, None, None]
    y = y * np.exp(sign * 2j * np.pi * ((j1 * k2) % n) / n)
    # p-point DFT over j1 for every (a, k2, r): Z[a, k2, k1, r] = sum_j1 F_p[k1, j1] y[a, k2, j1, r]
    if R == 1:
        z = np.matmul(y.reshape(A, m, p), dft_matrix(p, sign).T).reshape(A, m, p, 1)
    else:
        z = np.matmul(dft_matrix(p, sign), y)
    # output index k = k2 + m k1: order the axes (k1, k2)
    return np.ascontiguousarray(np.swapaxes(z, 1, 2)).reshape(A, n, R)


def fft(x: np.ndarray, axis: int = -1, sign: int = -1) -> np.ndarray:
    """Unnormalised complex DFT of x along `axis` (sign -1 forward, +1 inverse)."""
    x = np.ascontiguousarray(x, dtype=np.complex128)
    ax = axis % x.ndim
    A = int(np.prod(x.shape[:ax], dtype=np.int64))
    R = int(np.prod(x.shape[ax + 1:], dtype=np.int64))
    return _fft_mid(x.reshape(A, x.shape[ax], R), sign).reshape(x.shape)


def rfftn3(f: np.ndarray) -> np.ndarray:
    """Unnormalised forward real DFT over the last three axes: the full complex DFT along z
    of the real data, kept for kz = 0..nz/2, then complex DFTs along y and x."""
    nz = f.shape[-1]
    a = fft(np.asarray(f, dtype=np.complex128), axis=-1, sign=-1)[..., : nz // 2 + 1]
    a = fft(a, axis=-2, sign=-1)
    return fft(a, axis=-3, sign=-1)


def irfftn3(fhat: np.ndarray, shape) -> np.ndarray:
    """Inverse real DFT over the last three axes with the 1/(nx ny nz) normalisation.

    Complex inverse DFTs along x and y, then the real inverse along z: the half spectrum is
    extended by conjugate symmetry, Y[nz - k] = conj(Y[k]) for 0 < k < nz/2, and the real part
    of the complex inverse DFT is kept (which reads only Re Y[0] and Re Y[nz/2]).
    """
    nx, ny, nz = shape
    a = fft(fhat, axis=-3, sign=+1)
    a = fft(a, axis=-2, sign=+1)
    nh = nz // 2 + 1
    a = a[..., :nh]
    tail = np.conj(a[..., 1 : (nz + 1) // 2][..., ::-1])   # k = nz-1 .. nz/2+1 (or (nz+1)/2)
    full = np.concatenate([a, tail], axis=-1)
    return fft(full, axis=-1, sign=+1).real / float(nx * ny * nz)
