"""Seeded synthetic inputs for the pseudo-spectral Navier-Stokes workloads.

This module is shared by the CPU oracle, the tests and the benchmark.  It holds
only the definitions of the initial fields (closed-form Taylor-Green modes, a
random-phase turbulence field, a Rayleigh-Taylor density profile) and a
counter-based random number generator.  It does none of the method's arithmetic:
no right-hand side, no projection, no dealiasing, no time stepping.  Its one transform
is input construction: numpy's real FFT of the Rayleigh-Taylor density profile into the
half-spectrum layout (``rayleigh_taylor_hat``), for callers that take the initial state in
that layout (the oracle and the CUDA path each have their own transforms).

Spectral arrays use the half-spectrum layout ``[3][nx][ny][nz//2+1]`` (complex128,
component-major, kz contiguous) and the unnormalised forward DFT convention
``uhat_k = sum_x u(x) exp(-i k.x)`` on the grid ``x_j = L j / n``.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "splitmix64",
    "uniform01",
    "grid_axes",
    "signed_index",
    "taylor_green_3d",
    "taylor_green_2d",
    "taylor_green_3d_hat",
    "taylor_green_2d_hat",
    "random_solenoidal_hat",
    "random_complex_hat",
    "rayleigh_taylor_fields",
    "rayleigh_taylor_hat",
]

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(counter: np.ndarray, seed: int) -> np.ndarray:
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) evaluated at ``seed + gamma*(counter+1)``.

    Counter-based: output i depends only on (seed, counter[i]).  uint64 wraps mod 2^64.
    """
    c = np.asarray(counter, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + np.uint64(0x9E3779B97F4A7C15) * (c + np.uint64(1))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z & _MASK64


def uniform01(counter: np.ndarray, seed: int) -> np.ndarray:
    """Uniform doubles in (0, 1): the top 53 bits of SplitMix64, offset by half an ulp."""
    z = splitmix64(counter, seed)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def grid_axes(nx: int, ny: int, nz: int, lengths=(2 * np.pi, 2 * np.pi, 2 * np.pi)):
    """Grid point coordinates x_j = L j / n on [0, L) along each axis."""
    return tuple(L * np.arange(n) / n for n, L in zip((nx, ny, nz), lengths))


def signed_index(n: int) -> np.ndarray:
    """Signed integer mode numbers in FFT order: 0..n/2-1, -n/2..-1 (n even)."""
    return np.concatenate([np.arange(0, (n + 1) // 2), np.arange(-(n // 2), 0)])


# ----------------------------------------------------------------------------------
# Taylor-Green vortex (3D and its z-independent 2D variant), on [0, 2pi)^3.
# ----------------------------------------------------------------------------------

def taylor_green_3d(nx: int, ny: int, nz: int) -> np.ndarray:
    """Physical TG field u=(sin x cos y cos z, -cos x sin y cos z, 0), shape (3,nx,ny,nz)."""
    x, y, z = grid_axes(nx, ny, nz)
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
    u = np.zeros((3, nx, ny, nz))
    u[0] = np.sin(X) * np.cos(Y) * np.cos(Z)
    u[1] = -np.cos(X) * np.sin(Y) * np.cos(Z)
    return u


def taylor_green_2d(nx: int, ny: int, nz: int) -> np.ndarray:
    """Physical z-independent TG field u=(sin x cos y, -cos x sin y, 0)."""
    x, y, _ = grid_axes(nx, ny, nz)
    X, Y = np.meshgrid(x, y, indexing="ij")
    u = np.zeros((3, nx, ny, nz))
    u[0] = (np.sin(X) * np.cos(Y))[:, :, None]
    u[1] = (-np.cos(X) * np.sin(Y))[:, :, None]
    return u


def taylor_green_3d_hat(nx: int, ny: int, nz: int) -> np.ndarray:
    """Half-spectrum coefficients of the 3D TG field, written out from the trig identities.

    sin x = (e^{ix} - e^{-ix})/(2i), cos y = (e^{iy} + e^{-iy})/2, so with s_a = +-1:
    u_x has Fourier coefficient -i s_x/8 and u_y has +i s_y/8 at (s_x, s_y, s_z);
    the unnormalised DFT multiplies Fourier coefficients by nx*ny*nz.  Only s_z=+1 is
    stored in the half spectrum.
    """
    assert min(nx, ny, nz) >= 4
    uh = np.zeros((3, nx, ny, nz // 2 + 1), dtype=np.complex128)
    n3 = float(nx * ny * nz)
    for sx in (1, -1):
        for sy in (1, -1):
            ix, iy = sx % nx, sy % ny
            uh[0, ix, iy, 1] = n3 * (-1j * sx / 8.0)
            uh[1, ix, iy, 1] = n3 * (1j * sy / 8.0)
    return uh


def taylor_green_2d_hat(nx: int, ny: int, nz: int) -> np.ndarray:
    """Half-spectrum coefficients of the 2D TG field (kz = 0 plane only)."""
    assert min(nx, ny, nz) >= 4
    uh = np.zeros((3, nx, ny, nz // 2 + 1), dtype=np.complex128)
    n3 = float(nx * ny * nz)
    for sx in (1, -1):
        for sy in (1, -1):
            ix, iy = sx % nx, sy % ny
            uh[0, ix, iy, 0] = n3 * (-1j * sx / 4.0)
            uh[1, ix, iy, 0] = n3 * (1j * sy / 4.0)
    return uh


# ----------------------------------------------------------------------------------
# Random fields
# ----------------------------------------------------------------------------------

def _gaussian_pair(counter: np.ndarray, seed: int):
    """Two independent standard normals per counter (Box-Muller on two SplitMix64 draws)."""
    u1 = uniform01(2 * counter, seed)
    u2 = uniform01(2 * counter + 1, seed)
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)


def _hermitian_kz_planes(a: np.ndarray, nx: int, ny: int, nz: int) -> np.ndarray:
    """Make the kz=0 plane Hermitian: a(-kx,-ky,0) = conj(a(kx,ky,0)); zero the Nyquist rows.

    a has shape (..., nx, ny, nz//2+1).  Modes with kx=-nx/2, ky=-ny/2 or kz=nz/2 are set to
    zero so that every stored coefficient has a well-defined conjugate partner.
    """
    a = a.copy()
    a[..., nx // 2, :, :] = 0
    a[..., :, ny // 2, :] = 0
    a[..., :, :, nz // 2] = 0
    p = a[..., :, :, 0]
    ix = (-np.arange(nx)) % nx
    iy = (-np.arange(ny)) % ny
    mirror = np.conj(p[..., ix, :][..., :, iy])
    p = 0.5 * (p + mirror)
    p[..., 0, 0] = p[..., 0, 0].real
    a[..., :, :, 0] = p
    return a


def random_complex_hat(nx: int, ny: int, nz: int, seed: int, ncomp: int = 3) -> np.ndarray:
    """Complex Gaussian coefficients on every stored mode, Hermitian on kz=0 (no spectrum shape)."""
    nzh = nz // 2 + 1
    counter = np.arange(ncomp * nx * ny * nzh, dtype=np.uint64)
    g1, g2 = _gaussian_pair(counter, seed)
    a = (g1 + 1j * g2).reshape(ncomp, nx, ny, nzh)
    return _hermitian_kz_planes(a, nx, ny, nz)


def random_solenoidal_hat(nx: int, ny: int, nz: int, seed: int, k0: float = 4.0,
                          energy: float = 1.0) -> np.ndarray:
    """Random-phase divergence-free field with shell spectrum E(k) ~ k^4 exp(-2 (k/k0)^2).

    Construction: a random vector potential with |A_k| ~ exp(-(k/k0)^2) gives
    uhat = i k x A_k, which is orthogonal to k (divergence-free) and has |uhat| ~ k |A|, so
    the shell energy 4 pi k^2 |uhat|^2 ~ k^4 exp(-2 (k/k0)^2).  The field is scaled so that
    sum_k w_k |uhat_k|^2 / (2 (nx ny nz)^2) = energy, w_k = 1 on kz in {0, nz/2}, else 2.
    Domain [0, 2pi)^3, integer wavenumbers.
    """
    kx = signed_index(nx).astype(np.float64)[:, None, None]
    ky = signed_index(ny).astype(np.float64)[None, :, None]
    kz = np.arange(nz // 2 + 1, dtype=np.float64)[None, None, :]
    kmag = np.sqrt(kx * kx + ky * ky + kz * kz)
    A = random_complex_hat(nx, ny, nz, seed, 3) * np.exp(-(kmag / k0) ** 2)
    uh = np.empty_like(A)
    uh[0] = 1j * (ky * A[2] - kz * A[1])
    uh[1] = 1j * (kz * A[0] - kx * A[2])
    uh[2] = 1j * (kx * A[1] - ky * A[0])
    uh = _hermitian_kz_planes(uh, nx, ny, nz)
    w = np.full(nz // 2 + 1, 2.0)
    w[0] = 1.0
    if nz % 2 == 0:
        w[-1] = 1.0
    e = float(np.sum(w * np.abs(uh) ** 2)) / (2.0 * float(nx * ny * nz) ** 2)
    return uh * np.sqrt(energy / e)


def rayleigh_taylor_fields(nx: int, ny: int, nz: int, seed: int = 7, atwood: float = 0.5,
                           width: float = 0.05, amplitude: float = 1e-3, nmodes: int = 8):
    """Physical density deviation for a periodic two-interface Rayleigh-Taylor setup.

    Domain [0,2pi) x [0,2pi) x [0, Lz) with Lz = 2 pi nz/nx (same spacing on all axes).
    rho' = A [tanh((z - z1 - zeta)/w) - tanh((z - z2 - zeta)/w)] - A with z1 = Lz/4,
    z2 = 3 Lz/4: heavy fluid (rho' ~ +A) between the interfaces.  zeta(x, y) is a sum of
    cos(mx x + my y + phase) over 1 <= |mx|, |my| <= nmodes with seeded phases and total
    amplitude `amplitude`.  Velocity starts at rest.  Returns (rho, lengths).
    """
    lz = 2 * np.pi * nz / nx
    lengths = (2 * np.pi, 2 * np.pi * ny / nx, lz)
    x, y, z = grid_axes(nx, ny, nz, lengths)
    X, Y = np.meshgrid(x, y, indexing="ij")
    zeta = np.zeros((nx, ny))
    modes = [(mx, my) for mx in range(-nmodes, nmodes + 1) for my in range(-nmodes, nmodes + 1)
             if mx != 0 and my != 0]
    phases = 2 * np.pi * uniform01(np.arange(len(modes), dtype=np.uint64), seed)
    for (mx, my), ph in zip(modes, phases):
        zeta += np.cos(mx * X + my * Y + ph)
    zeta *= amplitude / np.sqrt(len(modes) / 2.0)
    z1, z2 = lz / 4, 3 * lz / 4
    Z = z[None, None, :]
    zt = zeta[:, :, None]
    rho = atwood * (np.tanh((Z - z1 - zt) / width) - np.tanh((Z - z2 - zt) / width)) - atwood
    return rho, lengths


def rayleigh_taylor_hat(nx: int, ny: int, nz: int, seed: int = 7, **kw):
    """The Rayleigh-Taylor initial state in the half-spectrum layout: [4][nx][ny][nz//2+1]
    complex128 with velocity zero and component 3 the unnormalised real DFT of the density
    deviation of ``rayleigh_taylor_fields`` (numpy.fft.rfftn; input construction only).
    Returns (state, lengths)."""
    rho, lengths = rayleigh_taylor_fields(nx, ny, nz, seed=seed, **kw)
    out = np.zeros((4, nx, ny, nz // 2 + 1), dtype=np.complex128)
    out[3] = np.fft.rfftn(rho)
    return out, lengths
