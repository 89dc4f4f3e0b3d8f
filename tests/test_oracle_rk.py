"""Pins for the oracle's Runge-Kutta pairs and step-size control (Section 2.2, Appendix A).

The tableaus are checked against the paper's printed fractions and against the order
conditions (exact rational arithmetic over all rooted trees), the integrators against
observed convergence orders on an ODE with a known solution, the controller against
hand-worked factors, and the whole adaptive driver against the exact decay of the
z-independent Taylor-Green flow.
"""
import math
import os
from fractions import Fraction as Fr

import numpy as np
import pytest

import synthetic as syn
from oracle import rk
from oracle import spectral as sp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_tableau(name):
    rows, b, bhat = [], None, None
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            head, _, rest = line.partition("|")
            vals = [Fr(v) for v in rest.split()]
            head = head.strip()
            if head == "b":
                b = vals
            elif head == "bhat":
                bhat = vals
            else:
                rows.append((Fr(head), vals))
    return rows, b, bhat


@pytest.mark.parametrize("tab,fname", [(rk.BS5, "tableau_bs5.txt"), (rk.DP5, "tableau_dp5.txt")])
def test_tableau_matches_appendix(tab, fname):
    rows, b, bhat = read_tableau(fname)
    assert [c for c, _ in rows] == list(tab.c)
    for (c, a), arow in zip(rows, tab.A):
        assert list(arow) == a
    assert list(tab.b) == b
    assert list(tab.bhat) == bhat


# ---- order conditions over rooted trees ------------------------------------------------

def rooted_trees(order):
    """All rooted trees with `order` nodes, as sorted tuples of child subtrees."""
    if order == 1:
        return [()]
    out = set()

    def partitions(n, maxpart):
        if n == 0:
            yield []
            return
        for p in range(min(n, maxpart), 0, -1):
            for rest in partitions(n - p, p):
                yield [p] + rest

    for parts in partitions(order - 1, order - 1):
        choices = [rooted_trees(p) for p in parts]

        def rec(i, acc):
            if i == len(parts):
                out.add(tuple(sorted(acc)))
                return
            for t in choices[i]:
                rec(i + 1, acc + [t])
        rec(0, [])
    return sorted(out)


def tree_order(t):
    return 1 + sum(tree_order(c) for c in t)


def density(t):
    """gamma(t) = |t| * prod gamma(children)."""
    g = tree_order(t)
    for c in t:
        g *= density(c)
    return g


def elementary_weight(t, A, s):
    """Vector Phi_i(t): product over children of (A Phi(child))_i, Phi(leaf) = 1."""
    v = [Fr(1)] * s
    for c in t:
        phic = elementary_weight(c, A, s)
        aphi = [sum((A[i][j] if j < len(A[i]) else 0) * phic[j] for j in range(s)) for i in range(s)]
        v = [v[i] * aphi[i] for i in range(s)]
    return v


def order_conditions_hold(tab, weights, p):
    s = tab.stages
    A = [list(r) for r in tab.A]
    for q in range(1, p + 1):
        for t in rooted_trees(q):
            phi = elementary_weight(t, A, s)
            if sum(w * x for w, x in zip(weights, phi)) != Fr(1, density(t)):
                return False
    return True


def test_tree_counts():
    # number of rooted trees with 1..6 nodes (OEIS A000081)
    assert [len(rooted_trees(n)) for n in range(1, 7)] == [1, 1, 2, 4, 9, 20]


@pytest.mark.parametrize("tab", [rk.RK4, rk.BS5, rk.DP5])
def test_row_sums_and_order_conditions(tab):
    for c, row in zip(tab.c, tab.A):
        assert sum(row, Fr(0)) == c
    assert order_conditions_hold(tab, tab.b, tab.order)
    assert not order_conditions_hold(tab, tab.b, tab.order + 1)
    if tab.bhat is not None:
        assert order_conditions_hold(tab, tab.bhat, tab.embedded_order)
        assert not order_conditions_hold(tab, tab.bhat, tab.embedded_order + 1)


@pytest.mark.parametrize("tab", [rk.BS5, rk.DP5])
def test_first_same_as_last(tab):
    assert list(tab.A[-1]) + [Fr(0)] == list(tab.b)
    assert tab.c[-1] == 1


def test_bs5_stability_polynomial_matches_exponential_to_order_5():
    # R(z) = 1 + sum_k b^T A^(k-1) 1 z^k; a fifth-order method has coefficient 1/k! for k <= 5
    tab = rk.BS5
    s = tab.stages
    A = [[(tab.A[i][j] if j < len(tab.A[i]) else Fr(0)) for j in range(s)] for i in range(s)]
    v = [Fr(1)] * s
    for k in range(1, 9):
        coeff_b = sum(bj * vj for bj, vj in zip(tab.b, v))
        coeff_bh = sum(bj * vj for bj, vj in zip(tab.bhat, v))
        if k <= 5:
            assert coeff_b == Fr(1, math.factorial(k))
        if k <= 4:
            assert coeff_bh == Fr(1, math.factorial(k))
        v = [sum(A[i][j] * v[j] for j in range(s)) for i in range(s)]
    assert coeff_b == 0                           # degree 7: an 8-stage FSAL pair's b ignores k8


# ---- observed convergence order ---------------------------------------------------------

def f_test(y):
    # rotation on the unit circle (nonlinear in form) plus a logistic component
    r2 = y[0] ** 2 + y[1] ** 2
    return np.array([-y[1] * r2, y[0] * r2, y[2] * (1 - y[2])])


def exact_test(t):
    y30 = 0.2
    return np.array([math.cos(t), math.sin(t), 1.0 / (1.0 + (1.0 / y30 - 1.0) * math.exp(-t))])


def run_fixed(tab, n, T=2.0, embedded=False):
    y = exact_test(0.0)
    h = T / n
    for _ in range(n):
        ynew, e, _ = rk.rk_attempt(f_test, y, h, tab)
        y = ynew - e if embedded else ynew
    return np.max(np.abs(y - exact_test(T)))


@pytest.mark.parametrize("tab,embedded,p", [(rk.RK4, False, 4), (rk.BS5, False, 5),
                                            (rk.BS5, True, 4), (rk.DP5, False, 5),
                                            (rk.DP5, True, 4)])
def test_observed_order(tab, embedded, p):
    e1 = run_fixed(tab, 10, embedded=embedded)
    e2 = run_fixed(tab, 20, embedded=embedded)
    e3 = run_fixed(tab, 40, embedded=embedded)
    o1, o2 = math.log2(e1 / e2), math.log2(e2 / e3)
    assert p - 0.3 < o2 < p + 0.6, (o1, o2)


def test_local_error_estimate_scales_like_h5():
    y = exact_test(0.0)
    es = []
    for h in (0.2, 0.1, 0.05):
        _, e, _ = rk.rk_attempt(f_test, y, h, rk.BS5)
        es.append(np.max(np.abs(e)))
    assert 4.5 < math.log2(es[1] / es[2]) < 5.5


# ---- controller -------------------------------------------------------------------------

def test_controller_factor_hand_worked():
    with open(os.path.join(GOLDEN, "controller_cases.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    assert len(rows) >= 10
    for err, after, fac, acc in rows:
        err = float(err)
        got = rk.controller_factor(err, bool(int(after)))
        assert abs(got - float(fac)) < 1e-14, (err, after, got, fac)
        assert (math.isfinite(err) and err <= 1.0) == bool(int(acc))


def test_adaptive_driver_invariants():
    # y' = lam y with a stiff-ish decay, large h0 to force rejections
    lam = -40.0

    def f(y):
        return lam * y
    res = rk.integrate(f, np.array([[1.0]]), 0.0, 1.0, "BS5_ADAPTIVE", h0=0.5, rtol=1e-6,
                       atol=1e-6, nmodes=1)
    assert res.status == "ok" and res.t == 1.0
    assert res.n_rej >= 1
    hist = res.history
    for i, (t, h, err, acc) in enumerate(hist):
        assert acc == (err <= 1.0)
        if i + 1 < len(hist):
            hn = hist[i + 1][1]
            if not acc:
                assert hn <= 0.8 * h + 1e-15           # retry is smaller
            elif i > 0 and not hist[i - 1][3]:
                assert hn <= h * (1 + 1e-15) or hist[i + 1][0] + hn == 1.0   # cap 1 after reject
    assert abs(hist[-1][0] + hist[-1][1] - 1.0) < 1e-15
    # 7 new RHS per attempt after the first (8 stages, first same as last)
    assert res.n_rhs == 8 + 7 * (len(hist) - 1)
    assert abs(res.u[0, 0] - math.exp(lam)) < 1e-5 * 50


@pytest.mark.parametrize("method,h0,tol", [("BS5_ADAPTIVE", 0.05, 1e-9), ("RK4", 0.01, None),
                                           ("BS5_FIXED", 0.05, 1e-9)])
def test_taylor_green_2d_decays_as_exp_minus_2_nu_t(method, h0, tol):
    n, nu, T = 16, 0.1, 1.0
    g = sp.Grid(n, n, n)
    u0 = syn.taylor_green_2d_hat(n, n, n)
    res = rk.integrate(lambda y: sp.rhs(g, y, nu), u0, 0.0, T, method, h0,
                       rtol=tol or 1e-6, atol=tol or 1e-6, nmodes=g.nmodes_half)
    assert res.t == T
    rel = np.max(np.abs(res.u - math.exp(-2 * nu * T) * u0)) / np.max(np.abs(u0))
    assert rel < 1e-9


def stability_poly(tab, weights, z):
    """R(z) = 1 + sum_k w^T A^(k-1) 1 z^k, evaluated with exact fractions then rounded."""
    s = tab.stages
    A = [[(tab.A[i][j] if j < len(tab.A[i]) else Fr(0)) for j in range(s)] for i in range(s)]
    v = [Fr(1)] * s
    zf = Fr(z)
    r, zk = Fr(1), Fr(1)
    for _ in range(s):
        zk *= zf
        r += sum(w * x for w, x in zip(weights, v)) * zk
        v = [sum(A[i][j] * v[j] for j in range(s)) for i in range(s)]
    return r


@pytest.mark.parametrize("nu,h,tol", [(0.5, 0.5, 1e-4), (0.2, 0.9, 1e-6), (1.0, 0.3, 1e-3)])
def test_error_norm_closed_form_tg2d(nu, h, tol):
    # For the z-independent TG flow f = -2 nu u exactly, so one BS5 attempt gives
    # u_new = R_b(z) u and e = (R_b(z) - R_bhat(z)) u with z = -2 nu h.  Each velocity
    # component has 4 stored modes of modulus a = N^3/4; the third component is zero, so
    # err = |dR| a / (atol + rtol max(a, |R_b| a)) * sqrt(4 / (N^2 (N/2+1))).
    n = 16
    g = sp.Grid(n, n, n)
    u0 = syn.taylor_green_2d_hat(n, n, n)
    u_new, e, _ = rk.rk_attempt(lambda y: sp.rhs(g, y, nu), u0, h, rk.BS5)
    err = rk.error_norm(u0, u_new, e, tol, tol, g.nmodes_half)
    z = -2 * nu * h
    Rb = float(stability_poly(rk.BS5, rk.BS5.b, z))
    dR = float(stability_poly(rk.BS5, rk.BS5.b, z) - stability_poly(rk.BS5, rk.BS5.bhat, z))
    a = n ** 3 / 4.0
    expect = abs(dR) * a / (tol + tol * max(a, abs(Rb) * a)) * math.sqrt(4.0 / g.nmodes_half)
    assert abs(err - expect) < 1e-9 * expect
    assert np.max(np.abs(u_new - Rb * u0)) < 1e-13 * a


@pytest.mark.parametrize("z,rtol", [(-0.5, 1e-4), (-0.36, 1e-6)])
def test_error_norm_pure_relative_tolerance(z, rtol):
    # atol = 0, a purely relative tolerance (Section 2.2.1 with the absolute part zero).  The
    # arrays are those of one BS5 step of the linear problem f = lambda u on a field whose
    # first two components hold 4 modes of modulus a and which is zero everywhere else (a
    # 2D Taylor-Green layout): u_new = R_b(z) u, e = (R_b(z) - R_bhat(z)) u exactly, z = h
    # lambda.  Every zero mode has sc = 0 and e = 0 and contributes nothing, so
    # err = |dR| / max(1, |R_b|) * sqrt(4 / nmodes) / rtol, independent of a.
    n = 16
    nmodes = n * n * (n // 2 + 1)
    Rb = float(stability_poly(rk.BS5, rk.BS5.b, z))
    dR = float(stability_poly(rk.BS5, rk.BS5.b, z) - stability_poly(rk.BS5, rk.BS5.bhat, z))
    expect = abs(dR) / (rtol * max(1.0, abs(Rb))) * math.sqrt(4.0 / nmodes)
    errs = []
    for a in (1.0, 1e6):
        u = np.zeros((3, n, n, n // 2 + 1), complex)
        for kx, ky in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
            u[0, kx, ky, 0] = -1j * a * np.sign(ky)
            u[1, kx, ky, 0] = 1j * a * np.sign(kx)
        err = rk.error_norm(u, Rb * u, dR * u, 0.0, rtol, nmodes)
        assert math.isfinite(err) and abs(err - expect) < 1e-12 * expect
        errs.append(err)
    assert abs(errs[1] - errs[0]) < 1e-12 * errs[0]
    # a nonzero error over a zero scale stays infinite (no tolerance can be met there)
    e2 = dR * u
    e2[2, 0, 0, 0] = 1e-3
    assert rk.error_norm(u, Rb * u, e2, 0.0, rtol, nmodes) == math.inf


def test_integrate_with_band_rescale_keeps_energy_and_refreshes_k1():
    # the Section 3.3.1 forcing after every accepted step: the energy stays at its initial value
    # and a first-same-as-last pair evaluates k_1 again for the rescaled state
    from oracle import diag
    n, nu, kf = 16, 0.02, 2.5
    g = sp.Grid(n, n, n)
    u0 = g.dealias(syn.random_solenoidal_hat(n, n, n, seed=6, k0=3.0))
    e0 = diag.energy(g, u0)
    energies = []
    res = rk.integrate(lambda u: sp.rhs(g, u, nu), u0, 0.0, 0.2, "BS5_ADAPTIVE", h0=0.01,
                       rtol=1e-6, atol=1e-6, nmodes=g.nmodes_half,
                       post_step=lambda a, b: sp.rescale_band(g, a, b, kf),
                       on_accept=lambda t, u, k: energies.append(diag.energy(g, u)))
    assert res.status == "ok" and res.n_acc >= 3
    assert max(abs(e - e0) for e in energies) < 1e-13 * e0
    assert res.n_rhs == 8 * res.n_acc + 7 * res.n_rej
    # without the rescale the same flow decays
    plain = rk.integrate(lambda u: sp.rhs(g, u, nu), u0, 0.0, 0.2, "BS5_ADAPTIVE", h0=0.01,
                         rtol=1e-6, atol=1e-6, nmodes=g.nmodes_half)
    assert diag.energy(g, plain.u) < e0 * (1 - 1e-3)
