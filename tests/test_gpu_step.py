"""Parity of the CUDA time integration (dns_step / dns_integrate) with the FP64 oracle:
Runge-Kutta stage sums, the embedded error norm and the step-size controller of Section 2.2.

FP64 bound: 1e-12 relative L2 on the state after 10 steps (rounding of ~70 right-hand sides,
each within 1e-13, accumulated linearly); decisions (accept/reject, counts) must agree exactly.
"""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import diag, rk
from oracle import spectral as sp
from tests.gpu_helpers import err_tolerance, lib_ready, rel_l2, rel_max, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    require_gpu()
    lib_ready()


def make(shape, uh, nu, precision="fp64", forcing=None, t0=0.0):
    from paper_1810_10197_gb300 import Dns
    d = Dns(*shape, nu=nu, precision=precision, forcing=forcing)
    d.set_state(to_dev(uh), t0)
    return d


def oracle_f(g, nu, forcing=None):
    return lambda y: sp.rhs(g, y, nu, forcing=forcing)


def test_single_bs5_attempt_matches_oracle():
    shape, nu, h = (32, 32, 32), 0.01, 0.05
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=12, k0=3.0))
    u_new, e, ks = rk.rk_attempt(oracle_f(g, nu), uh, h, rk.BS5)
    err = rk.error_norm(uh, u_new, e, 1e-6, 1e-6, g.nmodes_half)
    fac = rk.controller_factor(err, False)
    d = make(shape, uh, nu)
    info = d.step("BS5_ADAPTIVE", h, 1e-6, 1e-6)
    tol = err_tolerance(h, ks, e, rk.BS5, uh, u_new, 1e-6, 1e-6)
    assert abs(info.err - err) < tol * err
    assert bool(info.accepted) == (err <= 1)
    assert info.n_rhs == 8
    if info.accepted:
        assert rel_l2(d.get_state(), u_new) < 1e-13
        assert abs(info.h_next - h * fac) < (tol / 5 + 1e-15) * h * fac
        assert info.t == h


def test_pure_relative_tolerance_is_refused_for_adaptive_methods():
    # atol = 0 with an adaptive method: modes that the divergence-free constraint makes zero
    # up to rounding (u_x at kappa = (kx, 0, 0)) would carry an error and a scale that are
    # both rounding noise; the library refuses the call rather than run an arbitrary norm
    from paper_1810_10197_gb300.dns import DNS_ERR_ARG, DnsError
    shape, nu = (16, 16, 16), 0.01
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=21, k0=3.0))
    for method in ("BS5_ADAPTIVE", "DP5_ADAPTIVE"):
        d = make(shape, uh, nu)
        with pytest.raises(DnsError) as ex:
            d.step(method, 0.01, 1e-6, 0.0)
        assert ex.value.status == DNS_ERR_ARG and "atol" in str(ex.value)
        d.close()
    # the oracle's own norm on such a field: the modes where u_old = u_new = e = 0 exactly add
    # nothing (no NaN); a mode with rounding noise in e over a zero scale makes it infinite
    u_new, e, _ = rk.rk_attempt(oracle_f(g, nu), uh, 0.01, rk.BS5)
    err = rk.error_norm(uh, u_new, e, 0.0, 1e-6, g.nmodes_half)
    assert not math.isnan(err)


def test_rejected_attempt_keeps_state_and_shrinks_step():
    shape, nu = (16, 16, 16), 0.01
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=5, k0=3.0)) * 3
    h = 0.5
    u_new, e, ks = rk.rk_attempt(oracle_f(g, nu), uh, h, rk.BS5)
    err = rk.error_norm(uh, u_new, e, 1e-9, 1e-9, g.nmodes_half)
    assert err > 1
    d = make(shape, uh, nu)
    info = d.step("BS5_ADAPTIVE", h, 1e-9, 1e-9)
    assert not info.accepted and info.n_rej == 1 and info.t == 0.0
    tol = err_tolerance(h, ks, e, rk.BS5, uh, u_new, 1e-9, 1e-9)
    assert abs(info.err - err) < tol * err
    fac = rk.controller_factor(err, False)
    assert abs(info.h_next - h * fac) < (tol / 5 + 1e-15) * h * fac
    assert np.array_equal(d.get_state(), g.dealias(uh))


@pytest.mark.parametrize("method,h", [("RK4", 0.01), ("BS5_FIXED", 0.02)])
def test_fixed_steps_ten(method, h):
    shape, nu = (32, 32, 32), 0.01
    g = sp.Grid(*shape)
    uh = g.dealias(syn.taylor_green_3d_hat(*shape))
    T = 10 * h
    ref = rk.integrate(oracle_f(g, nu), uh, 0.0, T, method, h, nmodes=g.nmodes_half)
    d = make(shape, uh, nu)
    info = d.integrate(T, method, 1e-6, 1e-6, h0=h)
    assert info.n_acc == ref.n_acc == 10
    assert info.n_rhs == ref.n_rhs
    assert info.t == pytest.approx(T, abs=1e-15)
    assert rel_l2(d.get_state(), ref.u) < 1e-12


def test_taylor_green_config_bs5_adaptive_vs_oracle():
    # TG 32^3, nu = 0.01, t in [0, 1], rtol = atol = 1e-8, h0 = 0.01
    shape, nu = (32, 32, 32), 0.01
    g = sp.Grid(*shape)
    uh = g.dealias(syn.taylor_green_3d_hat(*shape))
    ref = rk.integrate(oracle_f(g, nu), uh, 0.0, 1.0, "BS5_ADAPTIVE", 0.01, 1e-8, 1e-8,
                       nmodes=g.nmodes_half)
    d = make(shape, uh, nu)
    info = d.integrate(1.0, "BS5_ADAPTIVE", 1e-8, 1e-8, h0=0.01)
    assert info.t == 1.0
    assert (info.n_acc, info.n_rej, info.n_rhs) == (ref.n_acc, ref.n_rej, ref.n_rhs)
    # err ~ 1e-8 |u| is resolved to ~1e-16/1e-8 relative, h_next to a fifth of that
    assert abs(info.h_next - ref.h_next) < 1e-7 * ref.h_next
    assert rel_l2(d.get_state(), ref.u) < 1e-12
    # RK4 with dt = 0.01 on the same flow
    ref4 = rk.integrate(oracle_f(g, nu), uh, 0.0, 1.0, "RK4", 0.01, nmodes=g.nmodes_half)
    d.set_state(to_dev(uh), 0.0)
    info4 = d.integrate(1.0, "RK4", h0=0.01)
    assert info4.n_rhs == ref4.n_rhs == 400
    assert rel_l2(d.get_state(), ref4.u) < 1e-12


def test_hit_forced_ten_adaptive_steps():
    shape, nu = (64, 64, 64), 1e-3
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=1, k0=4.0))
    forcing = (2.5, 0.2)
    f = oracle_f(g, nu, forcing)
    ref = rk.integrate(f, uh, 0.0, 1e9, "BS5_ADAPTIVE", 1e-3, 1e-6, 1e-6, nmodes=g.nmodes_half,
                       max_steps=10)
    d = make(shape, uh, nu, forcing=forcing)
    d.enqueue_attempts(10, "BS5_ADAPTIVE", 1e-6, 1e-6, t_end=1e9, h0=1e-3)
    info = d.info()
    assert (info.n_acc, info.n_rej) == (ref.n_acc, ref.n_rej)
    assert info.t == pytest.approx(ref.t, rel=1e-13)
    assert rel_l2(d.get_state(), ref.u) < 1e-12


def test_taylor_green_2d_decay_on_gpu():
    shape, nu = (32, 32, 32), 0.1
    uh = syn.taylor_green_2d_hat(*shape)
    d = make(shape, uh, nu)
    info = d.integrate(1.0, "BS5_ADAPTIVE", 1e-10, 1e-10, h0=0.05)
    assert info.t == 1.0
    assert rel_max(d.get_state(), math.exp(-2 * nu) * uh) < 1e-9


def test_diagnostics_match_oracle():
    shape, nu = (32, 32, 32), 0.02
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=6, k0=3.0))
    d = make(shape, uh, nu)
    E, O, eps = d.diagnostics()
    f = sp.rhs(g, uh, nu)
    assert E == pytest.approx(diag.energy(g, uh), rel=1e-13)
    assert O == pytest.approx(diag.enstrophy(g, uh), rel=1e-13)
    assert eps == pytest.approx(diag.dissipation(g, uh, f), rel=1e-12)
    assert eps == pytest.approx(2 * nu * O, rel=1e-12)


def test_fp32_mixed_ten_steps_error_is_small():
    shape, nu = (64, 64, 64), 1e-3
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=3, k0=4.0))
    ref = rk.integrate(oracle_f(g, nu), uh, 0.0, 1e9, "BS5_FIXED", 5e-3, nmodes=g.nmodes_half,
                       max_steps=10)
    d = make(shape, uh, nu, precision="fp32_mixed")
    d.enqueue_attempts(10, "BS5_FIXED", 1e-6, 1e-6, t_end=1e9, h0=5e-3)
    info = d.info()
    assert info.n_acc == 10
    assert rel_l2(d.get_state(), ref.u) < 1e-6


def test_step_underflow_and_nonfinite_statuses():
    from paper_1810_10197_gb300 import DnsError
    shape, nu = (16, 16, 16), 0.01
    uh = syn.random_solenoidal_hat(*shape, seed=2, k0=3.0)
    d = make(shape, uh, nu)
    with pytest.raises(DnsError) as ei:
        d.integrate(1.0, "BS5_ADAPTIVE", 1e-300, 1e-300, h0=0.1)
    assert ei.value.status in (5, 6)
    bad = uh.copy()
    bad[0, 1, 1, 1] = np.nan
    d2 = make(shape, bad, nu)
    st, info = d2.integrate(1.0, "BS5_ADAPTIVE", 1e-6, 1e-6, h0=0.1, max_rejects=3, check=False)
    assert st == 4 and info.n_rej == 4 and info.t == 0.0


@pytest.mark.parametrize("method,tol", [("DP5_ADAPTIVE", 1e-8), ("DP5_FIXED", 1e-6)])
def test_dp5_pair_matches_oracle(method, tol):
    # Appendix A's Dormand-Prince 5(4) pair through the same kernels (7 stages, FSAL)
    shape, nu = (32, 32, 32), 0.01
    g = sp.Grid(*shape)
    uh = g.dealias(syn.taylor_green_3d_hat(*shape) + 0.1 * syn.random_solenoidal_hat(*shape, seed=2, k0=3.0))
    ref = rk.integrate(oracle_f(g, nu), uh, 0.0, 0.5, method, 0.02, tol, tol, nmodes=g.nmodes_half)
    d = make(shape, uh, nu)
    info = d.integrate(0.5, method, tol, tol, h0=0.02)
    assert (info.n_acc, info.n_rej, info.n_rhs) == (ref.n_acc, ref.n_rej, ref.n_rhs)
    assert rel_l2(d.get_state(), ref.u) < 1e-12


def test_energy_spectrum_matches_oracle():
    shape = (48, 48, 48)
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=12, k0=4.0))
    d = make(shape, uh, 0.01)
    Ek = d.spectrum()
    ref = diag.energy_spectrum(g, uh)
    # the oracle's bincount also spans shells beyond the retained box (all zero here)
    assert len(Ek) >= len(np.trim_zeros(ref, "b"))
    assert np.all(ref[len(Ek):] == 0)
    assert np.max(np.abs(Ek - ref[:len(Ek)])) < 1e-12 * np.max(ref)
    assert abs(Ek.sum() - diag.energy(g, uh)) < 1e-12


def test_integrate_graph_matches_host_enqueued_attempts():
    # dns_integrate runs its attempts as one graph launch; the same attempts enqueued one by
    # one from the host (dns_enqueue_attempts) must give the identical state, bit for bit,
    # also after a tile change rebuilds the graph and when a second call continues the run
    shape, nu, tol = (32, 32, 32), 0.01, 1e-6
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=21, k0=3.0))
    a = make(shape, uh, nu)
    ia = a.integrate(0.2, "BS5_ADAPTIVE", tol, tol, h0=0.05)
    a.set_tiles(1, 1)
    ia2 = a.integrate(0.3, "BS5_ADAPTIVE", tol, tol, h0=0.0)
    b = make(shape, uh, nu)
    b.enqueue_attempts(ia.n_acc + ia.n_rej + 5, "BS5_ADAPTIVE", tol, tol, t_end=0.2, h0=0.05)
    ib = b.info()
    b.set_tiles(1, 1)
    b.enqueue_attempts(ia2.n_acc + ia2.n_rej - ib.n_acc - ib.n_rej + 5, "BS5_ADAPTIVE", tol, tol, t_end=0.3)
    ib2 = b.info()
    assert (ia.t, ia.n_acc, ia.n_rej) == (ib.t, ib.n_acc, ib.n_rej)
    assert (ia2.t, ia2.n_acc, ia2.n_rej, ia2.n_rhs) == (ib2.t, ib2.n_acc, ib2.n_rej, ib2.n_rhs)
    assert a.get_state().tobytes() == b.get_state().tobytes()
    # with per-kernel profiling on, the host loop gives the same result
    c = make(shape, uh, nu)
    c.profile_enable(True)
    c.integrate(0.2, "BS5_ADAPTIVE", tol, tol, h0=0.05)
    c.profile_enable(False)
    d = make(shape, uh, nu)
    d.integrate(0.2, "BS5_ADAPTIVE", tol, tol, h0=0.05)
    assert c.get_state().tobytes() == d.get_state().tobytes()


@pytest.mark.parametrize("index", [17, 40])
def test_injected_nan_is_rejected_and_the_run_recovers(index):
    # a one-shot NaN in right-hand side `index` (host-armed, no GPU fault): the attempt's err
    # is not finite, the controller rejects it with the smallest factor and the run finishes;
    # the oracle with the same fault in the same evaluation takes the same decisions
    shape, nu, tol, T = (32, 32, 32), 0.01, 1e-7, 0.3
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=8, k0=3.0))
    calls = [0]

    def f_inj(y):
        out = sp.rhs(g, y, nu)
        if calls[0] == index:
            out = out.copy()
            out[0, 0, 0, 0] = np.nan
        calls[0] += 1
        return out

    ref = rk.integrate(f_inj, uh, 0.0, T, "BS5_ADAPTIVE", 0.01, tol, tol, nmodes=g.nmodes_half)
    clean = rk.integrate(oracle_f(g, nu), uh, 0.0, T, "BS5_ADAPTIVE", 0.01, tol, tol, nmodes=g.nmodes_half)
    assert ref.status == "ok" and ref.n_rej >= clean.n_rej + 1
    assert any(not math.isfinite(e) for (_, _, e, _) in ref.history)
    d = make(shape, uh, nu)
    d.debug_inject(index)
    info = d.integrate(T, "BS5_ADAPTIVE", tol, tol, h0=0.01)
    assert info.t == T
    assert (info.n_acc, info.n_rej, info.n_rhs) == (ref.n_acc, ref.n_rej, ref.n_rhs)
    assert rel_l2(d.get_state(), ref.u) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed", "fp32"])
def test_injected_nan_in_a_carried_k1_ends_nonfinite(precision):
    # the very first evaluation is k_1 of u_0; a first-same-as-last pair reuses it after the
    # rejection, so every retry fails: DNS_ERR_NONFINITE after max_rejects, as in the oracle
    # (fp32: the NaN lands in the FP32 k slot)
    shape, nu = (16, 16, 16), 0.01
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=9, k0=3.0))
    d = make(shape, uh, nu, precision=precision)
    d.debug_inject(0)
    st, info = d.integrate(1.0, "BS5_ADAPTIVE", 1e-6, 1e-6, h0=0.05, max_rejects=3, check=False)
    assert st == 4 and info.n_rej == 4 and info.t == 0.0 and info.n_rhs == 8 + 3 * 7


@pytest.mark.parametrize("shape,kw", [((32, 48, 24), {}), ((16, 16, 16), {"dealias": "3/2"}),
                                      ((16, 16, 32), {"boussinesq": (0.01, 1.0)}), ((8, 8, 8), {})])
def test_host_state_upload_copies_the_retained_box(shape, kw):
    # dns_set_state from host memory copies only the retained modes (pitched copies into the
    # state buffer); the result equals the device path's gather bit for bit, whatever the
    # modes outside the box hold
    from paper_1810_10197_gb300 import Dns
    d = Dns(*shape, nu=0.01, **kw)
    nc = 4 if "boussinesq" in kw else 3
    rng = np.random.default_rng(sum(shape))
    full = rng.standard_normal((nc, shape[0], shape[1], shape[2] // 2 + 1)) \
        + 1j * rng.standard_normal((nc, shape[0], shape[1], shape[2] // 2 + 1))
    d.set_state(np.ascontiguousarray(full), 0.0)          # host pointer
    a = d.get_state()
    d.set_state(to_dev(full), 0.0)                        # device pointer
    b = d.get_state()
    assert a.tobytes() == b.tobytes()
    assert np.count_nonzero(a) > 0 and np.count_nonzero(a) < a.size
    d.close()
