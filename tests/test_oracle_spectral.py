"""Pins for the oracle's transforms and right-hand side (Section 2 of arXiv:1810.10197).

Each check compares the oracle with something it does not compute itself: brute-force
sums of the DFT definition, closed-form derivatives of trigonometric fields, an exact
mode-by-mode convolution (the alias-free product), and invariants of the equations.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import diag
from oracle import spectral as sp


def brute_dft_half(f, lengths=None):
    """uhat[mx,my,mz] = sum_x f(x) exp(-2 pi i (mx jx/nx + my jy/ny + mz jz/nz)), mz <= nz/2."""
    nx, ny, nz = f.shape[-3:]
    ex = np.exp(-2j * np.pi * np.outer(np.arange(nx), np.arange(nx)) / nx)
    ey = np.exp(-2j * np.pi * np.outer(np.arange(ny), np.arange(ny)) / ny)
    ez = np.exp(-2j * np.pi * np.outer(np.arange(nz // 2 + 1), np.arange(nz)) / nz)
    return np.einsum("ai,bj,ck,...ijk->...abc", ex, ey, ez, f)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 16, 17, 18, 24, 32, 36, 48, 96, 128, 192, 256, 384,
                               512, 768])
@pytest.mark.parametrize("sign", [-1, 1])
def test_own_fft_is_the_dft_sum(n, sign):
    # the oracle's Cooley-Tukey transform against the definition X[k] = sum_j x[j] w^(jk),
    # w = exp(sign 2 pi i / n), summed term by term; lengths above 16 exercise the recursion
    # (18 = 6 x 3, 768 = 16 x 16 x 3), and the transform runs along a middle axis, the last
    # axis and the first axis (the three data layouts of its code)
    from oracle import fft as offt
    rng = np.random.default_rng(n)
    x = rng.standard_normal((2, n, 3)) + 1j * rng.standard_normal((2, n, 3))
    jk = (np.arange(n)[:, None] * np.arange(n)[None, :]) % n
    w = np.exp(sign * 2j * np.pi * jk / n)
    ref = np.zeros_like(x)
    for k in range(n):
        ref[:, k, :] = np.sum(x * w[:, k][None, :, None], axis=1)
    tol = 1e-14 * max(1.0, np.log2(n)) * np.max(np.abs(ref))
    assert np.max(np.abs(offt.fft(x, axis=1, sign=sign) - ref)) <= tol
    xl = np.ascontiguousarray(np.moveaxis(x, 1, -1))
    assert np.max(np.abs(offt.fft(xl, axis=-1, sign=sign) - np.moveaxis(ref, 1, -1))) <= tol
    xf = np.ascontiguousarray(np.moveaxis(x, 1, 0))
    assert np.max(np.abs(offt.fft(xf, axis=0, sign=sign) - np.moveaxis(ref, 1, 0))) <= tol


@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 4, 8), (8, 6, 12), (12, 8, 6), (18, 24, 20)])
def test_forward_transform_is_unnormalised_dft(shape):
    rng = np.random.default_rng(1)
    f = rng.standard_normal((3,) + shape)
    g = sp.Grid(*shape)
    ref = brute_dft_half(f)
    got = g.to_spectral(f)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 4, 8), (8, 6, 12), (18, 24, 20)])
def test_inverse_transform_carries_one_over_n3(shape):
    rng = np.random.default_rng(2)
    f = rng.standard_normal(shape)
    g = sp.Grid(*shape)
    # the inverse of the brute-force forward DFT recovers f
    assert np.max(np.abs(g.to_physical(brute_dft_half(f)) - f)) < 1e-13
    # Parseval with half-spectrum weights: sum f^2 = sum_k w |fhat|^2 / N^3
    fh = g.to_spectral(f)
    lhs = np.sum(f * f)
    rhs_ = np.sum(g.weight[0] * np.abs(fh) ** 2) / g.n3
    assert abs(lhs - rhs_) < 1e-12 * lhs


def test_wavenumbers_spectral_derivative_exact_noncube():
    # domain [0,2pi) x [0,2pi) x [0,4pi): kappa_z = 2 pi m / 4 pi = m/2
    shape, L = (16, 12, 24), (2 * np.pi, 2 * np.pi, 4 * np.pi)
    g = sp.Grid(*shape, lengths=L)
    x, y, z = syn.grid_axes(*shape, L)
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
    f = np.sin(2 * X) * np.cos(3 * Y) * np.sin(1.5 * Z)
    fx = 2 * np.cos(2 * X) * np.cos(3 * Y) * np.sin(1.5 * Z)
    fy = -3 * np.sin(2 * X) * np.sin(3 * Y) * np.sin(1.5 * Z)
    fz = 1.5 * np.sin(2 * X) * np.cos(3 * Y) * np.cos(1.5 * Z)
    fh = g.to_spectral(f)
    for k, d in zip(g.kvec(), (fx, fy, fz)):
        assert np.max(np.abs(g.to_physical(1j * k * fh) - d)) < 1e-12


@pytest.mark.parametrize("n,K", [(8, 2), (12, 3), (16, 5), (32, 10), (64, 21), (96, 31), (128, 42),
                                 (256, 85), (512, 170)])
def test_two_thirds_cutoff(n, K):
    g = sp.Grid(n, n, n) if n <= 32 else None
    # largest K with 3K < n: products of two retained modes (|p|,|q| <= K) alias only onto
    # |m| >= n - 2K > K
    assert 3 * K < n <= 3 * (K + 1)
    if g is not None:
        assert g.cutoff == (K, K, K)
        assert not g.mask[:, :, n // 2].any()          # Nyquist never retained
        assert g.mask.sum() == (2 * K + 1) ** 2 * (K + 1)


def test_curl_of_taylor_green_closed_form():
    n = 16
    g = sp.Grid(n, n, n)
    uh = syn.taylor_green_3d_hat(n, n, n)
    w = g.to_physical(sp.curl_hat(g, uh))
    x, y, z = syn.grid_axes(n, n, n)
    X, Y, Z = np.meshgrid(x, y, z, indexing="ij")
    ref = np.stack([-np.cos(X) * np.sin(Y) * np.sin(Z),
                    -np.sin(X) * np.cos(Y) * np.sin(Z),
                    2 * np.sin(X) * np.sin(Y) * np.cos(Z)])
    assert np.max(np.abs(w - ref)) < 1e-13
    # the closed-form spectral TG coefficients equal the transform of the physical field
    assert np.max(np.abs(g.to_spectral(syn.taylor_green_3d(n, n, n)) - uh)) < 1e-12 * n ** 3


def full_spectrum(g, uh, cutoff=None):
    """Dict m -> coefficient vector over the retained box, expanded by Hermitian symmetry."""
    Kx, Ky, Kz = cutoff or g.cutoff
    out = {}
    for mx in range(-Kx, Kx + 1):
        for my in range(-Ky, Ky + 1):
            for mz in range(-Kz, Kz + 1):
                if mz >= 0:
                    out[(mx, my, mz)] = uh[:, mx % g.nx, my % g.ny, mz]
                else:
                    out[(mx, my, mz)] = np.conj(uh[:, (-mx) % g.nx, (-my) % g.ny, -mz])
    return out


def brute_force_rhs(g, uh, nu, cutoff=None):
    """Eq. (ufdef) with the nonlinear term as an exact convolution over retained modes.

    u(x) = (1/N^3) sum_p uhat_p e^{i p.x}; the DFT of u x omega at a retained k is
    (1/N^3) sum_{p+q=k} uhat_p x (i q x uhat_q) with no aliasing (3K < N).
    """
    L = g.lengths
    scale = [2 * np.pi / l for l in L]
    U = full_spectrum(g, uh, cutoff)
    W = {m: 1j * np.cross(np.array(m) * scale, v) for m, v in U.items()}
    Kx, Ky, Kz = g.cutoff
    f = np.zeros_like(uh)
    for (mx, my, mz), _ in U.items():
        if mz < 0:
            continue
        acc = np.zeros(3, dtype=complex)
        for p, up in U.items():
            q = (mx - p[0], my - p[1], mz - p[2])
            if q in W:
                acc += np.cross(up, W[q])
        acc /= g.n3
        kv = np.array((mx, my, mz)) * scale
        k2 = kv @ kv
        if k2 > 0:
            acc = acc - kv * (kv @ acc) / k2
        f[:, mx % g.nx, my % g.ny, mz] = acc - nu * k2 * U[(mx, my, mz)]
    return f


@pytest.mark.parametrize("shape,L", [((8, 8, 8), (2 * np.pi,) * 3),
                                     ((8, 12, 10), (2 * np.pi, 2 * np.pi, 2.5 * np.pi))])
def test_rhs_equals_brute_force_convolution(shape, L):
    g = sp.Grid(*shape, lengths=L)
    uh = g.dealias(syn.random_complex_hat(*shape, seed=5))
    f = sp.rhs(g, uh, nu=0.03)
    ref = brute_force_rhs(g, uh, 0.03)
    assert np.max(np.abs(f - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_taylor_green_2d_rhs_is_pure_decay():
    # for the z-independent TG flow u x omega is a gradient, so f = -2 nu uhat exactly
    n, nu = 16, 0.037
    g = sp.Grid(n, n, n)
    uh = syn.taylor_green_2d_hat(n, n, n)
    f = sp.rhs(g, uh, nu)
    assert np.max(np.abs(f + 2 * nu * uh)) < 1e-13 * np.max(np.abs(uh))


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 16, 8)])
def test_rhs_divergence_free_and_energy_identity(shape):
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=3, k0=3.0))
    nu = 0.02
    f = sp.rhs(g, uh, nu)
    scale = np.max(np.abs(f)) * np.sqrt(np.max(g.k2))
    assert diag.divergence_max(g, f) < 1e-13 * scale
    # semi-discrete energy identity: sum w Re(conj(u).f) = -nu sum w |kappa|^2 |u|^2
    lhs = np.sum(g.weight * np.real(np.conj(uh) * f))
    rhs_ = -nu * np.sum(g.weight * g.k2 * np.abs(uh) ** 2)
    assert abs(lhs - rhs_) < 1e-12 * abs(rhs_)
    # inviscid: the dealiased nonlinear term conserves energy
    f0 = sp.rhs(g, uh, 0.0)
    mag = np.sum(g.weight * np.abs(uh) * np.abs(f0))
    assert abs(np.sum(g.weight * np.real(np.conj(uh) * f0))) < 1e-13 * mag


def test_dealiasing_single_mode_product():
    # u = (0, 0, cos(a x)) has omega = (0, a sin(a x), 0); u x omega = (-a cos sin, 0, 0)
    # = (-(a/2) sin(2 a x), 0, 0).  With a = K the product mode 2K is outside the box and
    # must vanish (not alias back); with 2a <= K it must be reproduced exactly.
    n = 16
    g = sp.Grid(n, n, n)
    K = g.cutoff[0]
    x, _, _ = syn.grid_axes(n, n, n)
    for a in (K, K // 2):
        u = np.zeros((3, n, n, n))
        u[2] = np.cos(a * x)[:, None, None]
        nl = sp.nonlinear_hat(g, g.to_spectral(u))
        ref = np.zeros((3, n, n, n))
        if 2 * a <= K:
            ref[0] = (-(a / 2) * np.sin(2 * a * x))[:, None, None]
        assert np.max(np.abs(g.to_physical(nl) - ref)) < 1e-13 * max(a, 1)


def test_forcing_injects_constant_power():
    n = 16
    g = sp.Grid(n, n, n)
    uh = g.dealias(syn.random_solenoidal_hat(n, n, n, seed=9, k0=2.0))
    P = 0.37
    f = sp.rhs(g, uh, 0.0, forcing=(2.5, P))
    dEdt = np.sum(g.weight * np.real(np.conj(uh) * f)) / g.n3 ** 2
    assert abs(dEdt - P) < 1e-12 * P


def _decayed_pair(n=16, nu=0.05, h=0.05):
    """(u_old, u_new): one viscous BS5 step of a random solenoidal field (energy is lost)."""
    from oracle import rk
    g = sp.Grid(n, n, n)
    u0 = g.dealias(syn.random_solenoidal_hat(n, n, n, seed=4, k0=3.0))
    u1, _, _ = rk.rk_attempt(lambda u: sp.rhs(g, u, nu), u0, h, rk.BS5)
    return g, u0, u1


def test_band_rescale_restores_the_energy_lost_in_the_step():
    # Section 3.3.1: the low band is scaled so that the energy lost to diffusion is put back
    g, u0, u1 = _decayed_pair()
    e0, e1 = diag.energy(g, u0), diag.energy(g, u1)
    assert e1 < e0 * (1 - 1e-3)
    kf = 2.5
    u2 = sp.rescale_band(g, u0, u1, kf)
    assert abs(diag.energy(g, u2) - e0) < 1e-14 * e0
    band = np.broadcast_to((g.k2 > 0) & (g.k2 <= kf * kf) & g.mask, u1.shape)
    # outside the band nothing changes (bitwise); inside, one real factor > 1
    assert np.array_equal(u2[~band], u1[~band])
    nz = band & (np.abs(u1) > 1e-8 * np.max(np.abs(u1)))
    ratio = u2[nz] / u1[nz]
    assert np.max(np.abs(ratio.imag)) < 1e-15
    assert np.ptp(ratio.real) < 1e-14 and ratio.real[0] > 1.0


def test_band_rescale_special_cases():
    g, u0, u1 = _decayed_pair()
    # no energy lost: factor 1
    u2 = sp.rescale_band(g, u1, u1, 2.5)
    assert np.max(np.abs(u2 - u1)) <= 1e-15 * np.max(np.abs(u1))
    # an empty band (kf below the smallest wavenumber) leaves the very same state
    assert sp.rescale_band(g, u0, u1, 0.5) is u1
    # energy gained by more than the band holds: alpha^2 <= 0, state unchanged
    assert sp.rescale_band(g, 0.01 * u1, u1, 1.0) is u1


def test_boussinesq_hydrostatic_rest_state():
    # u = 0 with a density depending on z only: buoyancy is a pure gradient, so the velocity
    # right-hand side vanishes and the density only diffuses.
    shape, L = (8, 8, 16), (2 * np.pi, 2 * np.pi, 4 * np.pi)
    g = sp.Grid(*shape, lengths=L)
    _, _, z = syn.grid_axes(*shape, L)
    rho = np.broadcast_to(np.cos(z) + 0.3 * np.sin(2 * z), shape).copy()
    rh = g.dealias(g.to_spectral(rho))
    fu, fr = sp.rhs_boussinesq(g, np.zeros((3,) + rh.shape, complex), rh, 1e-3, 2e-3, 1.0)
    assert np.max(np.abs(fu)) < 1e-13 * np.max(np.abs(rh))
    assert np.max(np.abs(fr + 2e-3 * g.k2 * rh)) < 1e-13 * np.max(np.abs(rh))


def brute_force_boussinesq(g, uh, rh, nu, kappa, ri):
    """Eqs. (ufdefboussinesq), (rhofdefboussinesq) by exact convolution over retained modes.

    f_u = P(k)[(u x omega)^ - Ri rho_k e_z (k != 0)] - nu |k|^2 u_k,
    f_rho = -i k . (rho u)^ - kappa |k|^2 rho_k, with (rho u)^_k = (1/N^3) sum_{p+q=k} rho_p u_q.
    """
    scale = np.array([2 * np.pi / l for l in g.lengths])
    U = full_spectrum(g, uh)
    Rf = {m: v[0] for m, v in full_spectrum(g, rh[None]).items()}
    W = {m: 1j * np.cross(np.array(m) * scale, v) for m, v in U.items()}
    fu = np.zeros_like(uh)
    fr = np.zeros_like(rh)
    for (mx, my, mz) in U:
        if mz < 0:
            continue
        nl = np.zeros(3, dtype=complex)
        flux = np.zeros(3, dtype=complex)
        for p, up in U.items():
            q = (mx - p[0], my - p[1], mz - p[2])
            if q in W:
                nl += np.cross(up, W[q])
                flux += Rf[q] * up
        nl /= g.n3
        flux /= g.n3
        kv = np.array((mx, my, mz)) * scale
        k2 = kv @ kv
        if k2 > 0:
            nl[2] -= ri * Rf[(mx, my, mz)]
            nl = nl - kv * (kv @ nl) / k2
        ix, iy = mx % g.nx, my % g.ny
        fu[:, ix, iy, mz] = nl - nu * k2 * U[(mx, my, mz)]
        fr[ix, iy, mz] = -1j * (kv @ flux) - kappa * k2 * Rf[(mx, my, mz)]
    return fu, fr


def test_boussinesq_rhs_equals_brute_force_convolution():
    shape, L = (8, 8, 10), (2 * np.pi, 2 * np.pi, 2.5 * np.pi)
    g = sp.Grid(*shape, lengths=L)
    uh = g.dealias(syn.random_complex_hat(*shape, seed=31))
    rh = g.dealias(syn.random_complex_hat(*shape, seed=32, ncomp=1)[0])
    fu, fr = sp.rhs_boussinesq(g, uh, rh, 0.01, 0.02, 0.7)
    ru, rr = brute_force_boussinesq(g, uh, rh, 0.01, 0.02, 0.7)
    assert np.max(np.abs(fu - ru)) <= 1e-12 * np.max(np.abs(ru))
    assert np.max(np.abs(fr - rr)) <= 1e-12 * np.max(np.abs(rr))



@pytest.mark.parametrize("shape", [(8, 8, 8), (8, 12, 16)])
def test_pad32_rhs_equals_brute_force_convolution(shape):
    # the 3/2 padding rule keeps |m| <= N/2 - 1 and is alias-free: its result is the exact
    # convolution over the state's modes, truncated to those modes
    g = sp.Grid(*shape)
    K = tuple(n // 2 - 1 for n in shape)
    keep = (np.abs(g.mx) <= K[0]) & (np.abs(g.my) <= K[1]) & (g.mz <= K[2])
    uh = syn.random_complex_hat(*shape, seed=17) * keep
    f = sp.rhs_pad32(g, uh, 0.02)
    ref = brute_force_rhs(g, uh, 0.02, cutoff=K)
    assert np.max(np.abs(f - ref)) <= 1e-12 * np.max(np.abs(ref))
