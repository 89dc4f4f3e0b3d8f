"""Parity of the double-word form (DNS_FP32X2) with the FP64 oracle.

The transforms, the nonlinear term and the projection run on pairs of FP32 values.  A
double-word sum rounds with relative error at most u_dw = 2 u^2 = 2^-47 (7.1e-15, u = 2^-24)
of the operands' magnitude and a product at most 4 u^2; an FFT of length N adds
O(u_dw log2 N) normwise (log2 N <= 9 here), five axis passes and one product give a bound
near 50 u_dw = 3.6e-13 in the worst case; typical errors are a few u_dw.  Bounds used:
  * one right-hand side: 2e-13 relative max-norm (the FP64 path is held to 1e-13);
  * ten adaptive BS5 steps: decisions (accept/reject, counts) identical to the oracle's; the
    final time within 2e-10 relative (the embedded error is a cancellation that amplifies the
    right-hand side's rounding, see the test); the state, moved to the same time, within
    1e-12 relative L2, the FP64 path's bound.  Measured: FP64 2e-16, this form 9e-16.
    Compared without moving to the same time, the FP64 state differs by 1e-13 and this form's
    by about 7e-12: almost all of that is the state's change over the slightly different
    final time, not rounding of the state.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import rk
from oracle import spectral as sp
from tests.gpu_helpers import lib_ready, rel_l2, rel_max, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

DW_TOL = 2e-13


@pytest.fixture(scope="module", autouse=True)
def _lib():
    require_gpu()
    lib_ready()


def rhs(shape, uh, nu, **kw):
    from paper_1810_10197_gb300 import Dns
    d = Dns(*shape, nu=nu, precision="fp32x2", **kw)
    u = to_dev(uh)
    f = torch.empty_like(u)
    d.rhs(u, f)
    torch.cuda.synchronize()
    out = f.cpu().numpy()
    d.close()
    return out


@pytest.mark.parametrize("shape", [(32, 32, 32), (48, 48, 48), (64, 64, 64), (96, 96, 96), (128, 128, 128),
                                   (32, 64, 48), (192, 32, 64)])
def test_rhs_random_field(shape):
    g = sp.Grid(*shape)
    uh = syn.random_solenoidal_hat(*shape, seed=sum(shape) + 1, k0=max(2.0, shape[0] / 8))
    ref = sp.rhs(g, uh, 0.013)
    got = rhs(shape, uh, 0.013)
    assert rel_max(got, ref) < DW_TOL
    assert np.all(got[:, ~g.mask] == 0)


def test_rhs_forcing_and_noncube_domain():
    shape, L = (32, 48, 64), (2 * np.pi, 3.0, 5.0)
    g = sp.Grid(*shape, lengths=L)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=5, k0=3.0))
    ref = sp.rhs(g, uh, 0.02)
    assert rel_max(rhs(shape, uh, 0.02, lengths=L), ref) < DW_TOL
    g = sp.Grid(32, 32, 32)
    uh = g.dealias(syn.random_solenoidal_hat(32, 32, 32, seed=6, k0=3.0))
    ref = sp.rhs(g, uh, 0.01, forcing=(2.5, 0.3))
    assert rel_max(rhs((32, 32, 32), uh, 0.01, forcing=(2.5, 0.3)), ref) < DW_TOL


def test_rhs_three_halves_rule():
    shape = (32, 32, 32)
    g = sp.Grid(*shape)
    uh = syn.random_solenoidal_hat(*shape, seed=7, k0=4.0)
    ref = sp.rhs_pad32(g, uh, 0.01)
    assert rel_max(rhs(shape, uh, 0.01, dealias="3/2"), ref) < DW_TOL


def test_rhs_full_size_256():
    shape = (256, 256, 256)
    g = sp.Grid(*shape)
    uh = syn.random_solenoidal_hat(*shape, seed=1, k0=4.0)
    ref = sp.rhs(g, uh, 1e-3)
    assert rel_max(rhs(shape, uh, 1e-3), ref) < DW_TOL


def test_ten_adaptive_steps():
    from paper_1810_10197_gb300 import Dns
    shape, nu, tol = (64, 64, 64), 1e-3, 1e-6
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=1, k0=4.0))
    ref = rk.integrate(lambda y: sp.rhs(g, y, nu), uh, 0.0, 1e9, "BS5_ADAPTIVE", 1e-3, tol, tol,
                       nmodes=g.nmodes_half, max_steps=10)
    errs = {}
    for prec in ("fp64", "fp32x2"):
        d = Dns(*shape, nu=nu, precision=prec)
        d.set_state(to_dev(uh), 0.0)
        d.enqueue_attempts(10, "BS5_ADAPTIVE", tol, tol, t_end=1e9, h0=1e-3)
        info = d.info()
        assert (info.n_acc, info.n_rej, info.n_rhs) == (ref.n_acc, ref.n_rej, ref.n_rhs)
        # err is a cancellation: |e| ~ tol |u| while its terms are ~ h |k| ~ 0.1 |u|, so a
        # right-hand-side rounding eps moves err by ~ 0.05 eps 0.1 / tol = 5e3 eps, and h by a
        # fifth of that: 2e-11 per step at eps = 2e-14 (FP64: 5e-13 at 5e-16)
        assert info.t == pytest.approx(ref.t, rel=2e-10 if prec == "fp32x2" else 1e-12)
        # compare at the same time: move the oracle's state to the GPU's t to first order
        # (u + dt f(u)); what remains is the rounding of the state itself
        u_at = ref.u + (info.t - ref.t) * sp.rhs(g, ref.u, nu)
        errs[prec] = rel_l2(d.get_state(), u_at)
        d.close()
    print("ten-step relative L2 error:", errs)
    assert errs["fp64"] < 1e-12
    assert errs["fp32x2"] < 1e-12


def test_unsupported_sizes_are_refused():
    from paper_1810_10197_gb300 import Dns, DnsError
    for kw in ({"nx": 16}, {"nx": 32, "nz": 16}):
        with pytest.raises(DnsError) as ex:
            Dns(kw["nx"], 32, kw.get("nz", 32), nu=0.01, precision="fp32x2")
        assert ex.value.status == 9          # DNS_ERR_UNSUPPORTED


def test_boussinesq_rhs_and_steps():
    # Section 3.2's Boussinesq right-hand side in the double-word form: one evaluation at the
    # RHS bound, then 10 adaptive steps with identical decisions
    from paper_1810_10197_gb300 import Dns
    shape, nu, kap, ri = (32, 32, 64), 1e-2, 1e-2, 1.0
    L = (2 * np.pi, 2 * np.pi, 4 * np.pi)
    g = sp.Grid(*shape, lengths=L)
    u = g.dealias(syn.random_solenoidal_hat(*shape, seed=3, k0=3.0))
    r = g.dealias(syn.random_complex_hat(*shape, seed=4, ncomp=1)[0]) * 1e3
    st = np.concatenate([u, r[None]])
    fu, fr = sp.rhs_boussinesq(g, u, r, nu, kap, ri)
    ref = np.concatenate([fu, fr[None]])
    d = Dns(*shape, nu=nu, precision="fp32x2", boussinesq=(kap, ri), lengths=L)
    x = to_dev(st)
    f = torch.empty_like(x)
    d.rhs(x, f)
    torch.cuda.synchronize()
    assert rel_max(f.cpu().numpy(), ref) < DW_TOL

    def fb(y):
        a, b = sp.rhs_boussinesq(g, y[:3], y[3], nu, kap, ri)
        return np.concatenate([a, b[None]])
    tol = 1e-6
    res = rk.integrate(fb, g.dealias(st), 0.0, 1e9, "BS5_ADAPTIVE", 1e-3, tol, tol,
                       nmodes=g.nmodes_half, max_steps=10)
    d.set_state(x, 0.0)
    d.enqueue_attempts(10, "BS5_ADAPTIVE", tol, tol, t_end=1e9, h0=1e-3)
    info = d.info()
    assert (info.n_acc, info.n_rej, info.n_rhs) == (res.n_acc, res.n_rej, res.n_rhs)
    assert info.t == pytest.approx(res.t, rel=2e-10)
    u_at = res.u + (info.t - res.t) * fb(res.u)
    assert rel_l2(d.get_state(), u_at) < 1e-12
