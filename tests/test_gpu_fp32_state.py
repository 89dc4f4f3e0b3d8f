"""Stage sums, error norm and FP32 slots of the single-precision forms.

In both single-precision forms the k_j carry FP32 accuracy.  The fp32 form (DNS_FP32)
therefore stores k_j and the intermediate stage inputs in FP32 and forms the stage
increments sum_j (h a_ij) k_j and the embedded error e = h sum_j (b_j - bhat_j) k_j in FP32;
FP32-mixed keeps them FP64.  Both convert FP64 values to FP32 by an integer-bit conversion.
Checked here:
* the conversion against IEEE round-to-nearest (numpy float32) with its two stated
  differences: ties round away from zero, and magnitudes below the smallest normal float
  flush to a signed zero;
* the error norm's FP32 arithmetic against its FP64 arithmetic on the same attempt (the FP64
  arithmetic is taken for tolerances below 1e-30): at rtol 1e-3 the cancellation in e
  amplifies FP32 rounding (6e-8 of the terms) by h|k|/|e| ~ 1e2, bound 1e-4 relative;
* ten adaptive FP32-mixed steps against the oracle replaying the same step sizes (decisions
  need not match the oracle's own: the RHS's FP32 error moves err by a few percent at
  tolerance 1e-6), state within 1e-6 relative L2, as for fixed steps;
* the trace's dissipation rate, read from the carried k_1 (FP32 in the fp32 form), against
  the oracle within 1e-5;
* RK4 and DP5 in both forms (the other stage structures) against the oracle replaying the
  same steps.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import rk
from oracle import spectral as sp
from tests.gpu_helpers import lib_ready, rel_l2, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

FLT_MIN = float(np.finfo(np.float32).tiny)
FLT_MAX = float(np.finfo(np.float32).max)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    require_gpu()
    lib_ready()


def convert(x):
    from paper_1810_10197_gb300.dns import dns_debug_f32_from_f64
    xd = to_dev(np.asarray(x, dtype=np.float64))
    yd = torch.empty(xd.numel(), dtype=torch.float32, device="cuda")
    dns_debug_f32_from_f64(xd, yd)
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def test_conversion_matches_ieee_rounding_on_the_normal_range():
    rng = np.random.default_rng(11)
    n = 1 << 20
    x = rng.uniform(1.0, 2.0, n) * np.exp2(rng.integers(-126, 128, n).astype(np.float64))
    x *= np.where(rng.random(n) < 0.5, -1.0, 1.0)
    x = x[np.abs(x) <= FLT_MAX]
    got = convert(x)
    want = x.astype(np.float32)
    bits = x.view(np.uint64)
    tie = (bits & np.uint64(0x1FFFFFFF)) == np.uint64(0x10000000)
    assert np.array_equal(got[~tie], want[~tie])
    # a tie rounds away from zero
    assert np.all(np.abs(got[tie].astype(np.float64)) > np.abs(x[tie]))


def test_conversion_special_values():
    one_tie = 1.0 + 2.0 ** -24                 # halfway between 1 and 1 + 2^-23
    cases = [
        (0.0, 0.0), (-0.0, -0.0), (np.inf, np.inf), (-np.inf, -np.inf),
        (FLT_MIN, FLT_MIN), (-FLT_MIN, -FLT_MIN), (FLT_MIN * (1 - 2.0 ** -30), FLT_MIN),
        (FLT_MIN / 2, 0.0), (-1e-40, -0.0), (1e-300, 0.0), (5e-324, 0.0),
        (FLT_MAX, FLT_MAX), (3.5e38, np.inf), (-3.5e38, -np.inf), (1e300, np.inf),
        (FLT_MAX + 2.0 ** 103, np.inf),         # half an ulp above the largest float
        (one_tie, 1.0 + 2.0 ** -23), (-one_tie, -(1.0 + 2.0 ** -23)),
        (1.0 + 3 * 2.0 ** -24, 1.0 + 2.0 ** -22), (1.0 + 2.0 ** -25, 1.0), (np.pi, np.float32(np.pi)),
    ]
    x = np.array([c[0] for c in cases])
    got = convert(np.concatenate([x, [np.nan, -np.nan]]))
    for (xi, want), g in zip(cases, got):
        assert float(g) == want and np.signbit(g) == np.signbit(want), (xi, g, want)
    assert np.all(np.isnan(got[-2:]))


def attempt_err(shape, uh, nu, rtol, atol):
    from paper_1810_10197_gb300 import Dns
    d = Dns(*shape, nu=nu, precision="fp32")
    d.set_state(to_dev(uh), 0.0)
    info = d.step("BS5_ADAPTIVE", 2e-2, rtol, atol)
    d.close()
    return info


def test_error_norm_fp32_arithmetic_matches_fp64_arithmetic():
    shape, nu = (32, 32, 32), 0.01
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=5, k0=3.0))
    a = attempt_err(shape, uh, nu, 1e-3, 1e-20)     # FP32 arithmetic
    b = attempt_err(shape, uh, nu, 1e-3, 1e-31)     # FP64 arithmetic (atol below 1e-30)
    c = attempt_err(shape, uh, nu, 0.0, 1e-5)       # pure absolute tolerance: FP32 arithmetic
    d = attempt_err(shape, uh, nu, 1e-31, 1e-5)     # FP64 arithmetic
    assert 0.0 < a.err < 1e3 and 0.0 < c.err < 1e3
    assert a.err == pytest.approx(b.err, rel=1e-4)
    assert c.err == pytest.approx(d.err, rel=1e-4)


@pytest.mark.parametrize("shape,tiles", [((64, 64, 64), None), ((256, 24, 48), (4, 0)), ((256, 24, 48), (0, 0))])
@pytest.mark.parametrize("precision", ["fp32_mixed", "fp32"])
def test_single_precision_adaptive_steps_against_oracle(precision, shape, tiles):
    # ten adaptive attempts; the oracle replays the accepted step sizes from the attempt trace
    # in FP64, so the difference is the FP32 arithmetic alone (RHS, stage increments).  At
    # nx = 256 with and without the tensor-map x-inverse kernel (y argument bit 2), whose
    # stage input alternates between the two state buffers and the stage-input scratch (FP32
    # in the fp32 form)
    from paper_1810_10197_gb300 import Dns
    nu, tol = 1e-3, 1e-6
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=1, k0=4.0))
    d = Dns(*shape, nu=nu, precision=precision)
    if tiles is not None:
        d.set_tiles(*tiles)
    d.set_state(to_dev(uh), 0.0)
    d.set_trace(100)
    d.enqueue_attempts(10, "BS5_ADAPTIVE", tol, tol, t_end=1e9, h0=1e-3)
    info = d.info()
    tr = d.trace()
    assert info.n_acc >= 8 and len(tr) == 10
    u = uh.copy()
    for row in tr[tr[:, 3] > 0.5]:
        u = rk.rk_attempt(lambda y: sp.rhs(g, y, nu), u, float(row[1]), rk.TABLEAUS["BS5"], None)[0]
    assert float(np.sum(tr[tr[:, 3] > 0.5, 1])) == pytest.approx(info.t, rel=1e-14)
    assert rel_l2(d.get_state(), u) < 1e-6
    d.close()


def test_trace_dissipation_from_fp32_k_slots():
    # the attempt trace's dissipation rate reads the carried k_1, held in FP32 in this form
    from paper_1810_10197_gb300 import Dns
    from oracle import diag
    shape, nu = (32, 32, 32), 0.01
    g = sp.Grid(*shape)
    uh = g.dealias(syn.taylor_green_3d_hat(*shape) + 0.1 * syn.random_solenoidal_hat(*shape, seed=2, k0=3.0))
    d = Dns(*shape, nu=nu, precision="fp32")
    d.set_state(to_dev(uh), 0.0)
    d.set_trace(100, diagnostics=True)
    d.integrate(0.2, "BS5_ADAPTIVE", 1e-6, 1e-6, h0=0.01)
    tr = d.trace()
    u = d.get_state()
    assert tr[-1, 5] == pytest.approx(diag.energy(g, u), rel=1e-12)
    assert tr[-1, 7] == pytest.approx(diag.dissipation(g, u, sp.rhs(g, u, nu)), rel=1e-5)
    d.close()


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp32"])
@pytest.mark.parametrize("method,h0", [("RK4", 4e-3), ("DP5_ADAPTIVE", 1e-3)])
def test_single_precision_rk4_and_dp5_against_oracle(method, h0, precision):
    # the other stage structures through the FP32 slots: RK4 (one-term stage sums, four k
    # slots, no error norm) and DP5 (seven stages, six error terms); the oracle replays the
    # accepted step sizes in FP64
    from paper_1810_10197_gb300 import Dns
    shape, nu, tol = (48, 48, 48), 2e-3, 1e-6
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=4, k0=3.0))
    d = Dns(*shape, nu=nu, precision=precision)
    d.set_state(to_dev(uh), 0.0)
    d.set_trace(100)
    d.enqueue_attempts(8, method, tol, tol, t_end=1e9, h0=h0)
    tr = d.trace()
    acc = tr[tr[:, 3] > 0.5]
    assert len(acc) >= 6
    tab = rk.TABLEAUS["RK4" if method == "RK4" else "DP5"]
    u = uh.copy()
    for row in acc:
        u = rk.rk_attempt(lambda y: sp.rhs(g, y, nu), u, float(row[1]), tab, None)[0]
    assert rel_l2(d.get_state(), u) < 1e-6
    d.close()


@pytest.mark.parametrize("precision", ["fp32_mixed", "fp32"])
def test_single_precision_boussinesq_steps_against_oracle(precision):
    # the density component through the FP32 slots (fp32) or the FP64 ones (FP32-mixed): eight
    # adaptive attempts of a periodic Rayleigh-Taylor field, replayed by the oracle
    from paper_1810_10197_gb300 import Dns
    shape, nu, kap, ri, tol = (32, 32, 64), 1e-2, 1e-2, 1.0, 1e-6
    rho, L = syn.rayleigh_taylor_fields(*shape, seed=7, width=0.2, amplitude=1e-2)
    g = sp.Grid(*shape, lengths=L)
    Y = np.zeros((4, 32, 32, 33), complex)
    Y[3] = g.dealias(g.to_spectral(rho))
    Y[:3] = g.dealias(1e-3 * syn.random_solenoidal_hat(*shape, seed=5, k0=3.0))

    def fb(y):
        a, b = sp.rhs_boussinesq(g, y[:3], y[3], nu, kap, ri)
        return np.concatenate([a, b[None]])
    d = Dns(*shape, nu=nu, precision=precision, boussinesq=(kap, ri), lengths=L)
    d.set_state(to_dev(Y), 0.0)
    d.set_trace(100)
    d.enqueue_attempts(8, "BS5_ADAPTIVE", tol, tol, t_end=1e9, h0=1e-2)
    tr = d.trace()
    acc = tr[tr[:, 3] > 0.5]
    assert len(acc) >= 6
    u = Y.copy()
    for row in acc:
        u = rk.rk_attempt(fb, u, float(row[1]), rk.TABLEAUS["BS5"], None)[0]
    got = d.get_state()
    assert rel_l2(got[:3], u[:3]) < 1e-5 and rel_l2(got[3], u[3]) < 1e-6
    d.close()
