"""Kinetic energy, enstrophy and dissipation rate, written from Section 3.1 of arXiv:1810.10197.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 3.1 defines E_kin = ||uhat||^2 / (2 N^6) over all frequencies (the square of the norm
is dropped in the printed formula) and eps = -dE/dt = -(1/N^6) sum Re(conj(uhat) . f(uhat))
(the conjugate is dropped in the printed formula).  With the half spectrum each stored mode
0 < kz < nz/2 stands for itself and its conjugate (weight 2); kz = 0 and kz = nz/2 have
weight 1, which is the adjustment the paper mentions for the zero and Nyquist frequencies.
"""
from __future__ import annotations

import numpy as np

from .spectral import Grid


def energy(grid: Grid, uhat: np.ndarray) -> float:
    """E = sum_k w_k |uhat_k|^2 / (2 (nx ny nz)^2)."""
    return float(np.sum(grid.weight * np.abs(uhat) ** 2)) / (2.0 * grid.n3 ** 2)


def enstrophy(grid: Grid, uhat: np.ndarray) -> float:
    """Omega = sum_k w_k |kappa|^2 |uhat_k|^2 / (2 (nx ny nz)^2) = (1/2) <|omega|^2>."""
    return float(np.sum(grid.weight * grid.k2 * np.abs(uhat) ** 2)) / (2.0 * grid.n3 ** 2)


def dissipation(grid: Grid, uhat: np.ndarray, fhat: np.ndarray) -> float:
    """eps = -dE/dt = -sum_k w_k Re(conj(uhat_k) . f_k) / (nx ny nz)^2, f = d(uhat)/dt."""
    return -float(np.sum(grid.weight * np.real(np.conj(uhat) * fhat))) / grid.n3 ** 2


def divergence_max(grid: Grid, uhat: np.ndarray) -> float:
    """max_k |kappa . uhat_k| (zero for a solenoidal field)."""
    kx, ky, kz = grid.kvec()
    return float(np.max(np.abs(kx * uhat[0] + ky * uhat[1] + kz * uhat[2])))


def energy_spectrum(grid: Grid, uhat: np.ndarray) -> np.ndarray:
    """Shell-summed kinetic energy E(k) = sum_{|kappa| in shell k} w |uhat|^2 / (2 N^6),
    shell k = nearest integer to |kappa| (Section 3.3 plots this spectrum); sum_k E(k) = E."""
    shell = np.rint(np.sqrt(grid.k2)).astype(np.int64)
    e = grid.weight * np.sum(np.abs(uhat[:3]) ** 2, axis=0) / (2.0 * grid.n3 ** 2)
    return np.bincount(np.broadcast_to(shell, e.shape).ravel(), weights=e.ravel())
