"""Pins for the oracle's diagnostics (Section 3.1) and for the seeded synthetic inputs."""
import numpy as np
import pytest

import synthetic as syn
from oracle import diag
from oracle import spectral as sp


def test_taylor_green_energy_and_enstrophy_closed_form():
    # <u^2 + v^2>/2 = 1/8 for the TG field; every mode has |k|^2 = 3, so Omega = 3 E = 3/8
    n = 16
    g = sp.Grid(n, n, n)
    uh = syn.taylor_green_3d_hat(n, n, n)
    assert abs(diag.energy(g, uh) - 0.125) < 1e-15
    assert abs(diag.enstrophy(g, uh) - 0.375) < 1e-15
    # energy from the physical field directly
    u = syn.taylor_green_3d(n, n, n)
    assert abs(0.5 * np.mean(np.sum(u * u, axis=0)) - 0.125) < 1e-15


def test_unforced_dissipation_equals_two_nu_enstrophy():
    n, nu = 16, 0.013
    g = sp.Grid(n, n, n)
    uh = g.dealias(syn.random_solenoidal_hat(n, n, n, seed=4, k0=3.0))
    f = sp.rhs(g, uh, nu)
    eps = diag.dissipation(g, uh, f)
    assert abs(eps - 2 * nu * diag.enstrophy(g, uh)) < 1e-12 * eps


@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 8, 10)])
def test_random_solenoidal_field(shape):
    g = sp.Grid(*shape)
    uh = syn.random_solenoidal_hat(*shape, seed=11, k0=3.0)
    # divergence-free
    assert diag.divergence_max(g, uh) < 1e-12 * np.max(np.abs(uh)) * max(shape)
    # unit energy
    assert abs(diag.energy(g, uh) - 1.0) < 1e-13
    # Hermitian on the stored planes: a real field's transform reproduces the coefficients
    u = g.to_physical(uh)
    assert np.max(np.abs(g.to_spectral(u) - uh)) < 1e-10 * np.max(np.abs(uh))


def test_random_field_is_seeded_and_spectrum_peaks_near_k0():
    n, k0 = 48, 4.0
    a = syn.random_solenoidal_hat(n, n, n, seed=1, k0=k0)
    b = syn.random_solenoidal_hat(n, n, n, seed=1, k0=k0)
    c = syn.random_solenoidal_hat(n, n, n, seed=2, k0=k0)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    g = sp.Grid(n, n, n)
    shell = np.rint(np.sqrt(g.k2)).astype(int)
    e = np.bincount(shell.ravel(), weights=(g.weight * np.sum(np.abs(a) ** 2, axis=0)).ravel())
    kpeak = int(np.argmax(e[1:]) + 1)
    # E(k) ~ k^4 exp(-2 (k/k0)^2) peaks at k = k0
    assert abs(kpeak - k0) <= 1


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs of the published generator
    z = syn.splitmix64(np.arange(3, dtype=np.uint64), 0)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_rayleigh_taylor_profile():
    rho, L = syn.rayleigh_taylor_fields(16, 16, 32, seed=7)
    assert L[2] == pytest.approx(4 * np.pi)
    # heavy (+A) between the interfaces, light (-A) outside: (rho_h - rho_l)/(rho_h + rho_l) = A
    # about an ambient density of 1
    assert rho.max() <= 0.5 + 1e-12 and rho.min() >= -0.5 - 1e-12
    mid = rho[:, :, 16]
    edge = rho[:, :, 0]
    assert np.all(mid > 0.4) and np.all(edge < -0.4)


def test_energy_spectrum_sums_to_energy_and_places_tg_in_shell_2():
    n = 16
    g = sp.Grid(n, n, n)
    uh = syn.taylor_green_3d_hat(n, n, n)
    Ek = diag.energy_spectrum(g, uh)
    # every TG mode has |k| = sqrt(3) -> shell 2
    assert abs(Ek[2] - 0.125) < 1e-15 and abs(Ek.sum() - 0.125) < 1e-15
    r = g.dealias(syn.random_solenoidal_hat(n, n, n, seed=3, k0=3.0))
    assert abs(diag.energy_spectrum(g, r).sum() - diag.energy(g, r)) < 1e-13
