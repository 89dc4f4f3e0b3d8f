"""The 3/2 padding rule of Section 2.1.1 (dns_config.dealias = 1) against the oracle's
independent padded implementation, and the transform lengths 192, 384 and 768 on every axis
(elongated grids keep the oracle cheap).  FP64 bound 1e-13 as for the 2/3 rule."""
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


def keep32(g):
    return (np.abs(g.mx) < g.nx / 2) & (np.abs(g.my) < g.ny / 2) & (g.mz < g.nz / 2)


@pytest.mark.parametrize("shape", [(16, 16, 16), (32, 32, 32), (64, 32, 64), (128, 128, 128)])
@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed", "fp32"])
def test_pad32_rhs(shape, precision):
    from paper_1810_10197_gb300 import Dns
    g = sp.Grid(*shape)
    uh = syn.random_solenoidal_hat(*shape, seed=sum(shape), k0=3.0) * keep32(g)
    ref = sp.rhs_pad32(g, uh, 0.01)
    d = Dns(*shape, nu=0.01, precision=precision, dealias="3/2")
    u = to_dev(uh)
    f = torch.empty_like(u)
    d.rhs(u, f)
    torch.cuda.synchronize()
    got = f.cpu().numpy()
    assert rel_max(got, ref) < (1e-13 if precision == "fp64" else 2e-5)
    assert np.all(got[:, ~keep32(g)] == 0)          # Nyquist and beyond stay zero
    d.close()


def test_pad32_ten_adaptive_steps():
    from paper_1810_10197_gb300 import Dns
    shape, nu = (32, 32, 32), 0.01
    g = sp.Grid(*shape)
    uh = (syn.taylor_green_3d_hat(*shape) + 0.1 * syn.random_solenoidal_hat(*shape, seed=5, k0=3.0)) * keep32(g)
    ref = rk.integrate(lambda y: sp.rhs_pad32(g, y, nu), uh, 0.0, 1e9, "BS5_ADAPTIVE", 0.02, 1e-7, 1e-7,
                       nmodes=g.nmodes_half, max_steps=10)
    d = Dns(*shape, nu=nu, dealias="3/2")
    d.set_state(to_dev(uh), 0.0)
    d.enqueue_attempts(10, "BS5_ADAPTIVE", 1e-7, 1e-7, t_end=1e9, h0=0.02)
    info = d.info()
    assert (info.n_acc, info.n_rej) == (ref.n_acc, ref.n_rej)
    assert rel_l2(d.get_state(), ref.u) < 1e-12


@pytest.mark.parametrize("shape", [(768, 16, 16), (16, 768, 16), (16, 16, 768), (384, 24, 16),
                                   (16, 384, 32), (24, 16, 384), (192, 32, 24), (32, 192, 16), (16, 24, 192)])
def test_long_lines_2_3_rule(shape):
    from paper_1810_10197_gb300 import Dns
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_complex_hat(*shape, seed=3))
    ref = sp.rhs(g, uh, 0.005)
    d = Dns(*shape, nu=0.005)
    u = to_dev(uh)
    f = torch.empty_like(u)
    d.rhs(u, f)
    torch.cuda.synchronize()
    assert rel_max(f.cpu().numpy(), ref) < 1e-13
    d.close()
