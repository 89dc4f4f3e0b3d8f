"""Parity of the CUDA right-hand side (dns_rhs, Eq. ufdef) with the FP64 oracle.

FP64 bound: 1e-13 relative max-norm.  Each transform adds O(eps log2 N) relative error
(eps = 1.1e-16, log2 N <= 9, five axis passes and one product), i.e. ~1e-14; 1e-13 leaves a
factor of ten.  FP32-mixed bound: 2e-5 (eps_32 = 6e-8 times the same growth factor ~ 100).
"""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import diag
from oracle import spectral as sp
from tests.gpu_helpers import lib_ready, rel_max, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-13
FP32_TOL = 2e-5


def run_rhs(shape, uh, nu, precision="fp64", lengths=None, forcing=None, tiles=None):
    from paper_1810_10197_gb300 import Dns
    d = Dns(*shape, nu=nu, precision=precision, lengths=lengths, forcing=forcing)
    if tiles is not None:
        d.set_tiles(*tiles)
    u = to_dev(uh)
    f = torch.empty_like(u)
    d.rhs(u, f)
    torch.cuda.synchronize()
    out = f.cpu().numpy()
    d.close()
    return out


@pytest.fixture(scope="module", autouse=True)
def _lib():
    require_gpu()
    lib_ready()


@pytest.mark.parametrize("shape", [(8, 8, 8), (12, 12, 12), (16, 16, 16), (24, 24, 24), (32, 32, 32),
                                   (48, 48, 48), (64, 64, 64), (96, 96, 96), (128, 128, 128),
                                   (16, 24, 32), (32, 16, 8), (24, 48, 12)])
@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed", "fp32"])
def test_rhs_random_field(shape, precision):
    g = sp.Grid(*shape)
    uh = syn.random_solenoidal_hat(*shape, seed=sum(shape), k0=max(2.0, shape[0] / 8))
    nu = 0.013
    ref = sp.rhs(g, uh, nu)
    got = run_rhs(shape, uh, nu, precision)
    tol = FP64_TOL if precision == "fp64" else FP32_TOL
    assert rel_max(got, ref) < tol
    # outside the retained box the output is exactly zero
    assert np.all(got[:, ~g.mask] == 0)


@pytest.mark.parametrize("shape", [(32, 256, 64), (16, 256, 48), (24, 256, 32),
                                   (32, 128, 64), (24, 128, 48), (16, 128, 32), (32, 128, 256)])
@pytest.mark.parametrize("precision", ["fp32_mixed", "fp32"])
def test_rhs_y_pass_variants_at_ny_256_and_128(shape, precision):
    # y-pass variant 2 (tensor-map tiles, register-resident transforms) applies at ny = 256
    # and 128 with an even number of retained kz planes (Mz = 22, 16, 86; the shapes with
    # nz = 32 have Mz = 11 and run variant 0); every variant against the oracle
    g = sp.Grid(*shape)
    uh = syn.random_solenoidal_hat(*shape, seed=sum(shape) + 1, k0=4.0)
    ref = sp.rhs(g, uh, 0.011)
    for tiles in ((0, 0), (1, 4), (2, 0), (2, 4)):
        got = run_rhs(shape, uh, 0.011, precision, tiles=tiles)
        assert rel_max(got, ref) < FP32_TOL, tiles
        assert np.all(got[:, ~g.mask] == 0)


@pytest.mark.parametrize("shape,forcing", [((256, 32, 64), None), ((256, 24, 48), (2.5, 0.1))])
@pytest.mark.parametrize("precision", ["fp32_mixed", "fp32"])
def test_rhs_nx_256_boxes(shape, forcing, precision):
    # the benchmark's x-line length on thin boxes, forcing included, against the oracle
    g = sp.Grid(*shape)
    uh = syn.random_solenoidal_hat(*shape, seed=sum(shape) + 2, k0=4.0)
    ref = sp.rhs(g, uh, 0.013, forcing=forcing)
    for tiles in ((0, 0), (4, 0)):     # k_p1, the tensor-map x-inverse kernel
        got = run_rhs(shape, uh, 0.013, precision, forcing=forcing, tiles=tiles)
        assert rel_max(got, ref) < FP32_TOL, tiles
        assert np.all(got[:, ~g.mask] == 0)


def test_rhs_non_solenoidal_and_noncube_domain():
    shape, L = (16, 16, 32), (2 * np.pi, 2 * np.pi, 4 * np.pi)
    g = sp.Grid(*shape, lengths=L)
    uh = syn.random_complex_hat(*shape, seed=3)
    ref = sp.rhs(g, uh, 0.02)
    got = run_rhs(shape, uh, 0.02, lengths=L)
    assert rel_max(got, ref) < FP64_TOL


def test_rhs_with_constant_power_forcing():
    shape = (32, 32, 32)
    g = sp.Grid(*shape)
    uh = syn.random_solenoidal_hat(*shape, seed=8, k0=3.0)
    ref = sp.rhs(g, uh, 1e-3, forcing=(2.5, 0.1))
    got = run_rhs(shape, uh, 1e-3, forcing=(2.5, 0.1))
    assert rel_max(got, ref) < FP64_TOL


def test_rhs_taylor_green_2d_pure_decay():
    shape, nu = (32, 32, 32), 0.05
    uh = syn.taylor_green_2d_hat(*shape)
    got = run_rhs(shape, uh, nu)
    assert rel_max(got, -2 * nu * uh) < FP64_TOL


def test_rhs_empty_field_is_zero():
    shape = (16, 16, 16)
    got = run_rhs(shape, np.zeros((3, 16, 16, 9), complex), 0.1)
    assert np.all(got == 0)


def test_rhs_full_size_256_against_oracle():
    # the benchmark's grid: TG 256^3 at nu = 1/1600 plus a random field (full oracle RHS)
    shape = (256, 256, 256)
    g = sp.Grid(*shape)
    for uh, nu in ((syn.taylor_green_3d_hat(*shape), 1 / 1600),
                   (syn.random_solenoidal_hat(*shape, seed=1, k0=4.0), 1e-3)):
        ref = sp.rhs(g, uh, nu)
        got = run_rhs(shape, uh, nu)
        assert rel_max(got, ref) < FP64_TOL
        # the single-precision forms at this size, with the register-resident z pass (tile
        # code 4) and with the shared-memory one (code 0), the y passes in each variant (2:
        # tensor-map tiles) and the x-inverse pass in each (y argument + 4: tensor-map tiles)
        for precision in ("fp32_mixed", "fp32"):
            for tiles in ((0, 4), (1, 0), (2, 4), (6, 4), (4, 0)):
                got = run_rhs(shape, uh, nu, precision, tiles=tiles)
                assert rel_max(got, ref) < FP32_TOL, (precision, tiles)


@pytest.fixture(scope="module")
def field_512():
    g = sp.Grid(512, 512, 512)
    return g, g.dealias(syn.random_solenoidal_hat(512, 512, 512, seed=2, k0=4.0))


# (divergence bound relative to max|f| |k|max, energy-identity bound relative to
# sum w |u| |f|): FP64 rounding ~1e-16 and double-word ~1e-14 grown by the transforms;
# FP32 ~6e-8 grown by the same factor (the RHS parity bound 2e-5 allows ~300x)
BOUNDS_512 = {"fp64": (1e-12, 1e-12), "fp32x2": (1e-11, 1e-11), "fp32_mixed": (2e-5, 2e-5),
              "fp32": (2e-5, 2e-5)}


@pytest.mark.parametrize("precision", ["fp64", "fp32x2", "fp32_mixed", "fp32"])
def test_rhs_full_size_512_properties(field_512, precision):
    # at 512^3 the oracle is too slow for a full comparison; check what holds at any size:
    # divergence-free output and the semi-discrete energy identity sum w Re(conj(u) f) =
    # -nu sum w |k|^2 |u|^2 (the nonlinear part conserves energy), in every form.
    g, uh = field_512
    nu = 1e-3
    got = run_rhs((512, 512, 512), uh, nu, precision=precision)
    bdiv, ben = BOUNDS_512[precision]
    scale = np.max(np.abs(got)) * math.sqrt(float(np.max(g.k2 * g.mask)))
    assert diag.divergence_max(g, got) < bdiv * scale
    lhs = np.sum(g.weight * np.real(np.conj(uh) * got))
    rhs_ = -nu * np.sum(g.weight * g.k2 * np.abs(uh) ** 2)
    size = np.sum(g.weight * np.abs(uh) * np.abs(got))
    assert abs(lhs - rhs_) < ben * size, (precision, lhs, rhs_, size)
    if precision == "fp64":      # and against the dissipation itself
        assert abs(lhs - rhs_) < 1e-11 * abs(rhs_)
