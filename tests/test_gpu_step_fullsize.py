"""Step parity at the benchmark's grid: one Bogacki-Shampine 5(4) attempt at 256^3 and ten
adaptive attempts at 128^3, against the FP64 oracle (Section 2.2, Appendix A).

At these sizes the error norm's sums run over millions of modes and the state magnitudes
span more decades than on the small grids of test_gpu_step.py, so the stage sums, the
Newton-refined square root and reciprocal of the norm (and their range branches) and the
controller are exercised at the size the benchmark runs.  Each oracle right-hand side at
256^3 takes about ten seconds on one host core.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import rk
from oracle import spectral as sp
from tests.gpu_helpers import err_tolerance, lib_ready, rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    require_gpu()
    lib_ready()


def oracle_f(g, nu):
    return lambda y: sp.rhs(g, y, nu)


@pytest.mark.parametrize("flow", ["taylor_green", "random"])
def test_one_bs5_attempt_at_256(flow):
    from paper_1810_10197_gb300 import Dns
    n, nu, tol = 256, 1.0 / 1600.0, 1e-6
    g = sp.Grid(n, n, n)
    if flow == "taylor_green":
        uh, h = g.dealias(syn.taylor_green_3d_hat(n, n, n)), 0.05
    else:
        uh, h = g.dealias(syn.random_solenoidal_hat(n, n, n, seed=9, k0=4.0)), 2e-3
    u_new, e, ks = rk.rk_attempt(oracle_f(g, nu), uh, h, rk.BS5)
    err = rk.error_norm(uh, u_new, e, tol, tol, g.nmodes_half)
    fac = rk.controller_factor(err, False)
    d = Dns(n, nu=nu)
    d.set_state(to_dev(uh), 0.0)
    info = d.step("BS5_ADAPTIVE", h, tol, tol)
    etol = err_tolerance(h, ks, e, rk.BS5, uh, u_new, tol, tol)
    assert abs(info.err - err) < etol * err, (flow, info.err, err, etol)
    assert bool(info.accepted) == (err <= 1)
    assert info.n_rhs == 8
    assert abs(info.h_next - h * fac) < (etol / 5 + 1e-15) * h * fac
    if info.accepted:
        assert info.t == h
        assert rel_l2(d.get_state(), u_new) < 1e-13
    else:
        assert np.array_equal(d.get_state(), uh)
    d.close()


def test_ten_adaptive_attempts_at_128():
    from paper_1810_10197_gb300 import Dns
    n, nu, tol = 128, 1e-3, 1e-6
    g = sp.Grid(n, n, n)
    uh = g.dealias(syn.random_solenoidal_hat(n, n, n, seed=4, k0=4.0))
    ref = rk.integrate(oracle_f(g, nu), uh, 0.0, 1e9, "BS5_ADAPTIVE", 5e-3, tol, tol,
                       nmodes=g.nmodes_half, max_steps=10)
    d = Dns(n, nu=nu)
    d.set_state(to_dev(uh), 0.0)
    d.enqueue_attempts(10, "BS5_ADAPTIVE", tol, tol, t_end=1e9, h0=5e-3)
    info = d.info()
    assert (info.n_acc, info.n_rej, info.n_rhs) == (ref.n_acc, ref.n_rej, ref.n_rhs)
    assert info.t == pytest.approx(ref.t, rel=1e-13)
    assert rel_l2(d.get_state(), ref.u) < 1e-12
    d.close()
