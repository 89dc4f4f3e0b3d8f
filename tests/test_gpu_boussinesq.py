"""Parity of the CUDA Boussinesq right-hand side and integration (Section 3.2, Eqs.
ufdefboussinesq / rhofdefboussinesq) with the FP64 oracle.  Same bounds as the
Navier-Stokes parity tests: 1e-13 (FP64) / 2e-5 (FP32-mixed) on one right-hand side,
1e-12 relative L2 on the state after 10 steps with identical accept/reject decisions."""
import numpy as np
import pytest

import synthetic as syn
from oracle import rk
from oracle import spectral as sp
from tests.gpu_helpers import lib_ready, rel_l2, rel_max, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    require_gpu()
    lib_ready()


def oracle_f(g, nu, kappa, ri):
    def f(Y):
        fu, fr = sp.rhs_boussinesq(g, Y[:3], Y[3], nu, kappa, ri)
        return np.concatenate([fu, fr[None]])
    return f


def state(shape, L, seed):
    g = sp.Grid(*shape, lengths=L)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=seed, k0=3.0))
    rh = g.dealias(syn.random_complex_hat(*shape, seed=seed + 1, ncomp=1)) * (0.1 * float(np.prod(shape)))
    return g, np.concatenate([uh, rh])


def gpu_rhs(shape, L, Y, nu, kappa, ri, precision="fp64", tiles=None):
    from paper_1810_10197_gb300 import Dns
    d = Dns(*shape, nu=nu, precision=precision, lengths=L, boussinesq=(kappa, ri))
    if tiles is not None:
        d.set_tiles(*tiles)
    y = to_dev(Y)
    f = torch.empty_like(y)
    d.rhs(y, f)
    torch.cuda.synchronize()
    out = f.cpu().numpy()
    d.close()
    return out


@pytest.mark.parametrize("shape,L", [((8, 8, 8), None), ((16, 16, 32), (2 * np.pi, 2 * np.pi, 4 * np.pi)),
                                     ((24, 32, 48), (2 * np.pi, 8 * np.pi / 3, 4 * np.pi)),
                                     ((64, 64, 128), (2 * np.pi, 2 * np.pi, 4 * np.pi))])
@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed", "fp32"])
def test_boussinesq_rhs(shape, L, precision):
    Lr = L or (2 * np.pi,) * 3
    g, Y = state(shape, Lr, 40 + shape[0])
    ref = oracle_f(g, 1e-3, 2e-3, 1.0)(Y)
    got = gpu_rhs(shape, Lr, Y, 1e-3, 2e-3, 1.0, precision)
    tol = 1e-13 if precision == "fp64" else 2e-5
    assert rel_max(got[:3], ref[:3]) < tol
    assert rel_max(got[3], ref[3]) < tol


@pytest.mark.parametrize("shape", [(16, 256, 64), (16, 128, 64)])
@pytest.mark.parametrize("precision", ["fp32_mixed", "fp32"])
def test_boussinesq_rhs_y_pass_tensor_map(shape, precision):
    # y-pass variant 2 at ny = 256 and 128: seven inverse planes (u, omega, rho) and six
    # forward ones
    L = (2 * np.pi, 2 * np.pi, 4 * np.pi)
    g, Y = state(shape, L, 77)
    ref = oracle_f(g, 1e-3, 2e-3, 1.0)(Y)
    got = gpu_rhs(shape, L, Y, 1e-3, 2e-3, 1.0, precision, tiles=(2, 0))
    assert rel_max(got[:3], ref[:3]) < 2e-5
    assert rel_max(got[3], ref[3]) < 2e-5


def test_boussinesq_hydrostatic_rest_state():
    shape, L = (16, 16, 32), (2 * np.pi, 2 * np.pi, 4 * np.pi)
    g = sp.Grid(*shape, lengths=L)
    _, _, z = syn.grid_axes(*shape, L)
    rho = np.broadcast_to(np.cos(z) + 0.3 * np.sin(2 * z), shape).copy()
    Y = np.zeros((4, 16, 16, 17), complex)
    Y[3] = g.dealias(g.to_spectral(rho))
    got = gpu_rhs(shape, L, Y, 1e-3, 2e-3, 1.0)
    assert np.max(np.abs(got[:3])) < 1e-13 * np.max(np.abs(Y[3]))


def test_rayleigh_taylor_ten_adaptive_steps():
    # periodic two-interface RT (Atwood 0.5, width 0.05 scaled to the grid), at rest
    from paper_1810_10197_gb300 import Dns
    shape = (32, 32, 64)
    rho, L = syn.rayleigh_taylor_fields(*shape, seed=7, width=0.2, amplitude=1e-2)
    g = sp.Grid(*shape, lengths=L)
    Y = np.zeros((4, 32, 32, 33), complex)
    Y[3] = g.dealias(g.to_spectral(rho))
    nu = kappa = 1e-3
    ref = rk.integrate(oracle_f(g, nu, kappa, 1.0), Y, 0.0, 1e9, "BS5_ADAPTIVE", 0.01, 1e-6, 1e-6,
                       nmodes=g.nmodes_half, max_steps=10)
    d = Dns(*shape, nu=nu, lengths=L, boussinesq=(kappa, 1.0))
    d.set_state(to_dev(Y), 0.0)
    d.enqueue_attempts(10, "BS5_ADAPTIVE", 1e-6, 1e-6, t_end=1e9, h0=0.01)
    info = d.info()
    assert (info.n_acc, info.n_rej) == (ref.n_acc, ref.n_rej)
    assert info.t == pytest.approx(ref.t, rel=1e-12)
    got = d.get_state()
    assert got.shape == (4, 32, 32, 33)
    assert rel_l2(got[:3], ref.u[:3]) < 1e-12
    assert rel_l2(got[3], ref.u[3]) < 1e-12
