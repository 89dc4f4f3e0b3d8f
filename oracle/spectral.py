"""Pseudo-spectral right-hand side, written from Section 2 of arXiv:1810.10197.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Plain FP64 numpy; the DFT is the
oracle's own Cooley-Tukey transform (oracle/fft.py), pinned against the brute-force DFT sum.

Conventions (readings of the paper, each listed in the design notes):
  * Domain [0, L_x) x [0, L_y) x [0, L_z), default L = 2 pi; wavenumber kappa_a = 2 pi m / L_a
    with integer mode numbers m.
  * Spectral arrays use the half spectrum of a real DFT along z (the paper takes the real
    DFT "in the first direction"; the axis is a layout choice): shape (ncomp, nx, ny, nz//2+1).
  * The forward DFT is unnormalised, uhat_k = sum_x u(x) exp(-i k.x); the inverse carries
    1/(nx ny nz).  This follows from E = ||uhat||^2 / (2 N^6) (Section 3.1).
  * Dealiasing: the 2/3 truncation rule.  A mode is retained iff |m_a| <= K_a for every axis,
    K_a = floor((n_a - 1)/3), the largest K with 3K < n (so quadratic products do not alias
    onto retained modes).  Nyquist modes are never retained.  The paper's own runs used
    the 3/2 padding rule (Section 2.1.1); both rules give alias-free retained modes.
  * Leray projection P(kappa) = I - kappa kappa^T / |kappa|^2, with P(0) = I.  Eq. (ufdef)
    prints the pressure term as "i k (k . N)/|k|^2"; the factor i is dimensionally
    inconsistent and is read as a typo (with it the result would not be divergence-free).
"""
from __future__ import annotations

import numpy as np

from . import fft as _fft


class Grid:
    """Wavenumbers, 2/3 mask and transforms for an nx x ny x nz periodic grid."""

    def __init__(self, nx: int, ny: int, nz: int, lengths=(2 * np.pi, 2 * np.pi, 2 * np.pi)):
        self.shape = (nx, ny, nz)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.nzh = nz // 2 + 1
        self.lengths = tuple(float(L) for L in lengths)
        mx = np.fft.fftfreq(nx, d=1.0 / nx)
        my = np.fft.fftfreq(ny, d=1.0 / ny)
        mz = np.arange(self.nzh, dtype=np.float64)
        # integer mode numbers (FFT order) and physical wavenumbers
        self.mx = mx[:, None, None]
        self.my = my[None, :, None]
        self.mz = mz[None, None, :]
        self.kx = (2 * np.pi / self.lengths[0]) * self.mx
        self.ky = (2 * np.pi / self.lengths[1]) * self.my
        self.kz = (2 * np.pi / self.lengths[2]) * self.mz
        self.k2 = self.kx ** 2 + self.ky ** 2 + self.kz ** 2
        self.cutoff = tuple((n - 1) // 3 for n in self.shape)
        Kx, Ky, Kz = self.cutoff
        self.mask = ((np.abs(self.mx) <= Kx) & (np.abs(self.my) <= Ky) & (self.mz <= Kz))
        # half-spectrum weights: a stored mode 0 < mz < nz/2 stands for itself and its conjugate
        w = np.full(self.nzh, 2.0)
        w[0] = 1.0
        if nz % 2 == 0:
            w[-1] = 1.0
        self.weight = w[None, None, :]
        self.n3 = float(nx * ny * nz)
        # number of stored frequencies, the divisor of the error norm (Section 2.2.1)
        self.nmodes_half = nx * ny * self.nzh

    # ---- transforms -------------------------------------------------------------------
    def to_physical(self, fhat: np.ndarray) -> np.ndarray:
        """Inverse real DFT over the last three axes (carries 1/(nx ny nz))."""
        return _fft.irfftn3(fhat, self.shape)

    def to_spectral(self, f: np.ndarray) -> np.ndarray:
        """Unnormalised forward real DFT over the last three axes."""
        return _fft.rfftn3(f)

    def dealias(self, fhat: np.ndarray) -> np.ndarray:
        """2/3 rule: zero every mode outside the retained box."""
        return fhat * self.mask

    def kvec(self):
        return (self.kx, self.ky, self.kz)


def cross(a, b):
    """Pointwise cross product of two 3-vectors given as sequences/arrays of components."""
    return np.stack([a[1] * b[2] - a[2] * b[1],
                     a[2] * b[0] - a[0] * b[2],
                     a[0] * b[1] - a[1] * b[0]])


def curl_hat(grid: Grid, uhat: np.ndarray) -> np.ndarray:
    """Spectral vorticity omega_hat = i kappa x uhat (Section 2, omega = curl u)."""
    k = grid.kvec()
    return 1j * cross([np.broadcast_to(c, uhat.shape[1:]) for c in k], uhat)


def leray(grid: Grid, nhat: np.ndarray) -> np.ndarray:
    """P(kappa) nhat = nhat - kappa (kappa . nhat)/|kappa|^2, identity at kappa = 0."""
    kx, ky, kz = grid.kvec()
    k2 = np.where(grid.k2 == 0, 1.0, grid.k2)
    kdotn = (kx * nhat[0] + ky * nhat[1] + kz * nhat[2]) / k2
    out = np.empty_like(nhat)
    out[0] = nhat[0] - kx * kdotn
    out[1] = nhat[1] - ky * kdotn
    out[2] = nhat[2] - kz * kdotn
    return out


def nonlinear_hat(grid: Grid, uhat: np.ndarray) -> np.ndarray:
    """Dealiased transform of u x omega, evaluated in physical space (Section 2.1)."""
    u = grid.to_physical(uhat)
    w = grid.to_physical(curl_hat(grid, uhat))
    return grid.dealias(grid.to_spectral(cross(u, w)))


def band_energy(grid: Grid, uhat: np.ndarray, kf: float) -> float:
    """Energy held in 0 < |kappa| <= kf, with the half-spectrum weights."""
    band = (grid.k2 > 0) & (grid.k2 <= kf * kf) & grid.mask
    return float(np.sum(grid.weight * band * np.abs(uhat) ** 2)) / (2.0 * grid.n3 ** 2)


def forcing_hat(grid: Grid, uhat: np.ndarray, kf: float, power: float) -> np.ndarray:
    """Constant-power forcing F_k = (P / (2 E_f)) uhat_k on 0 < |kappa| <= kf.

    The paper rescales the low band after every step (Section 3.3.1); as a right-hand-side
    term the same injection is written so that dE/dt gains exactly P.
    """
    band = (grid.k2 > 0) & (grid.k2 <= kf * kf) & grid.mask
    ef = band_energy(grid, uhat, kf)
    if ef <= 0.0:
        return np.zeros_like(uhat)
    return (power / (2.0 * ef)) * band * uhat


def rescale_band(grid: Grid, u_old: np.ndarray, u_new: np.ndarray, kf: float) -> np.ndarray:
    """The paper's deterministic forcing (Section 3.3.1), applied after an accepted step.

    The modes 0 < |kappa| <= kf of the new state are multiplied by one factor alpha, chosen so
    that the energy the step lost is put back: E(rescaled) = E(u_old).  With E_f the band
    energy of u_new this gives alpha^2 = 1 + (E(u_old) - E(u_new)) / E_f.  Without band energy,
    or when alpha^2 <= 0, the new state is returned unchanged.
    """
    def e(u):
        return float(np.sum(grid.weight * grid.mask * np.abs(u) ** 2)) / (2.0 * grid.n3 ** 2)

    ef = band_energy(grid, u_new, kf)
    if not ef > 0.0:
        return u_new
    a2 = 1.0 + (e(u_old) - e(u_new)) / ef
    if not a2 > 0.0:
        return u_new
    band = (grid.k2 > 0) & (grid.k2 <= kf * kf) & grid.mask
    return np.where(band, np.sqrt(a2) * u_new, u_new)


def rhs(grid: Grid, uhat: np.ndarray, nu: float, forcing=None) -> np.ndarray:
    """Right-hand side of Eq. (ufdef): f = P(kappa)[u x omega]^ - nu |kappa|^2 uhat (+ forcing).

    The state space is the set of dealiased fields: the input is truncated to the retained
    box and the output is zero outside it.  `forcing` is None or (kf, power).
    """
    yhat = grid.dealias(uhat)
    f = leray(grid, nonlinear_hat(grid, yhat)) - nu * grid.k2 * yhat
    if forcing is not None:
        kf, power = forcing
        f = f + forcing_hat(grid, yhat, kf, power)
    return grid.dealias(f)


def rhs_boussinesq(grid: Grid, uhat: np.ndarray, rhohat: np.ndarray, nu: float, kappa: float,
                   ri: float):
    """Boussinesq right-hand sides, Eqs. (ufdefboussinesq) and (rhofdefboussinesq).

    du/dt = P(kappa)[u x omega - Ri rho e_z]^ - nu |kappa|^2 uhat
    drho/dt = -i kappa . (rho u)^ - kappa_d |kappa|^2 rhohat
    The buoyancy term enters inside the projection; its kappa = 0 mode is dropped (a mean
    body force is balanced by the mean pressure gradient in a periodic box).  The printed
    "i k" factor in the pressure term is read as in Eq. (ufdef).
    """
    yhat = grid.dealias(uhat)
    rh = grid.dealias(rhohat)
    u = grid.to_physical(yhat)
    w = grid.to_physical(curl_hat(grid, yhat))
    rho = grid.to_physical(rh)
    nl = grid.dealias(grid.to_spectral(cross(u, w)))
    buoy = -ri * rh * (grid.k2 > 0)
    nl[2] = nl[2] + buoy
    fu = grid.dealias(leray(grid, nl) - nu * grid.k2 * yhat)
    flux = grid.dealias(grid.to_spectral(rho[None] * u))
    kx, ky, kz = grid.kvec()
    frho = -1j * (kx * flux[0] + ky * flux[1] + kz * flux[2]) - kappa * grid.k2 * rh
    return fu, grid.dealias(frho)


def rhs_pad32(grid: Grid, uhat: np.ndarray, nu: float) -> np.ndarray:
    """Eq. (ufdef) with the 3/2 padding rule of Section 2.1.1.

    The state has N frequencies per axis; u and omega are zero-padded to 3N/2 frequencies,
    transformed to the (3N/2)^3 grid, u x omega is formed there and transformed back, and
    the highest frequencies are truncated to leave N per axis.  The Nyquist modes (which the
    paper's footnote reports as a source of spurious imaginary parts) are kept at zero, so
    the state has |m| <= N/2 - 1.  Normalisation stays that of the N-grid DFT.
    """
    nx, ny, nz = grid.shape
    P = (3 * nx // 2, 3 * ny // 2, 3 * nz // 2)
    keep = (np.abs(grid.mx) < nx / 2) & (np.abs(grid.my) < ny / 2) & (grid.mz < nz / 2)
    y = uhat * keep

    def pad(a):
        out = np.zeros(a.shape[:-3] + (P[0], P[1], P[2] // 2 + 1), dtype=complex)
        ix = np.concatenate([np.arange(nx // 2), np.arange(P[0] - nx // 2, P[0])])
        iy = np.concatenate([np.arange(ny // 2), np.arange(P[1] - ny // 2, P[1])])
        src_x = np.concatenate([np.arange(nx // 2), np.arange(nx - nx // 2, nx)])
        src_y = np.concatenate([np.arange(ny // 2), np.arange(ny - ny // 2, ny)])
        out[..., ix[:, None], iy[None, :], :nz // 2 + 1] = a[..., src_x[:, None], src_y[None, :], :]
        return out

    def unpad(a):
        ix = np.concatenate([np.arange(nx // 2), np.arange(P[0] - nx // 2, P[0])])
        iy = np.concatenate([np.arange(ny // 2), np.arange(P[1] - ny // 2, P[1])])
        src_x = np.concatenate([np.arange(nx // 2), np.arange(nx - nx // 2, nx)])
        src_y = np.concatenate([np.arange(ny // 2), np.arange(ny - ny // 2, ny)])
        out = np.zeros(a.shape[:-3] + (nx, ny, nz // 2 + 1), dtype=complex)
        out[..., src_x[:, None], src_y[None, :], :] = a[..., ix[:, None], iy[None, :], :nz // 2 + 1]
        return out

    r = (P[0] * P[1] * P[2]) / float(nx * ny * nz)
    u = _fft.irfftn3(pad(y), P) * r
    w = _fft.irfftn3(pad(curl_hat(grid, y)), P) * r
    nl = unpad(_fft.rfftn3(cross(u, w))) / r * keep
    return (leray(grid, nl) - nu * grid.k2 * y) * keep
