"""Learned and PI step-size controllers, the network kernels and the attempt trace.

* network forward and gradient (dns_mlp_forward / dns_mlp_loss_grad, bf16 weights, FP32
  arithmetic) against the FP64 oracle with the same bf16-rounded weights: 1e-5 / 1e-4
  relative (FP32 accumulation over 16..64 terms and up to 128 samples);
* training on the GPU lowers the loss;
* PI and MLP controllers on the device make the same accept/reject decisions as the oracle;
* the trace's diagnostics match the oracle's (Section 3.1);
* the gain of the trained network over the Section 2.2.1 controller on a Rayleigh-Taylor run
  (trained on Taylor-Green and forced-turbulence trajectories) is measured and reported.
"""
import math

import numpy as np
import pytest

import synthetic as syn
from oracle import diag, mlp, rk
from oracle import spectral as sp
from tests.gpu_helpers import lib_ready, rel_l2, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    require_gpu()
    lib_ready()


def dev32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_network_forward_and_gradient_match_oracle():
    from paper_1810_10197_gb300.dns import dns_mlp_forward, dns_mlp_loss_grad
    rng = np.random.default_rng(5)
    p = (mlp.init_params(2) + 0.05 * rng.standard_normal(mlp.N_PARAMS)).astype(np.float32)
    X = rng.standard_normal((100, 16)).astype(np.float32)
    t = rng.standard_normal(100).astype(np.float32)
    pr = mlp.round_bf16(p)
    y_ref, _ = mlp.forward(pr, X.astype(np.float64))
    L_ref, g_ref = mlp.loss_and_grad(pr, X.astype(np.float64), t.astype(np.float64))
    pd, xd, td = dev32(p), dev32(X), dev32(t)
    y = torch.empty(100, dtype=torch.float32, device="cuda")
    g = torch.empty(mlp.N_PARAMS, dtype=torch.float32, device="cuda")
    L = torch.empty(1, dtype=torch.float32, device="cuda")
    assert dns_mlp_forward(pd, xd, y) == 0
    assert dns_mlp_loss_grad(pd, xd, td, g, L) == 0
    torch.cuda.synchronize()
    assert np.max(np.abs(y.cpu().numpy() - y_ref)) < 1e-5 * np.max(np.abs(y_ref))
    assert abs(L.item() - L_ref) < 1e-5 * L_ref
    gg = g.cpu().numpy()
    assert np.max(np.abs(gg - g_ref)) < 1e-4 * np.max(np.abs(g_ref))
    # parameters are not modified by the gradient call
    assert np.array_equal(pd.cpu().numpy(), p)


def test_training_on_gpu_lowers_the_loss():
    from paper_1810_10197_gb300 import learned
    rng = np.random.default_rng(0)
    X = rng.standard_normal((2000, 16)).astype(np.float32)
    T = (np.tanh(X[:, 0] - 0.5 * X[:, 3]) + 0.3 * X[:, 5]).astype(np.float32)
    p, hist = learned.train(X, T, steps=1500, lr=2e-3, seed=1)
    assert np.all(np.isfinite(hist))
    assert hist[-100:].mean() < 0.1 * hist[:20].mean()


def run_pair(controller, params=None, shape=(32, 32, 32), nu=0.01, T=1.0, tol=1e-8):
    from paper_1810_10197_gb300 import Dns
    g = sp.Grid(*shape)
    uh = g.dealias(syn.taylor_green_3d_hat(*shape))
    ctl = controller if controller != "MLP" else ("MLP", params)
    ref = rk.integrate(lambda y: sp.rhs(g, y, nu), uh, 0.0, T, "BS5_ADAPTIVE", 0.01, tol, tol,
                       nmodes=g.nmodes_half, controller=ctl)
    d = Dns(*shape, nu=nu)
    d.set_state(to_dev(uh), 0.0)
    if controller == "MLP":
        d.set_controller("MLP", dev32(params))
    else:
        d.set_controller(controller)
    info = d.integrate(T, "BS5_ADAPTIVE", tol, tol, h0=0.01)
    return ref, info, d


def test_pi_controller_matches_oracle():
    ref, info, d = run_pair("PI")
    assert (info.n_acc, info.n_rej, info.n_rhs) == (ref.n_acc, ref.n_rej, ref.n_rhs)
    assert abs(info.h_next - ref.h_next) < 1e-7 * ref.h_next
    assert rel_l2(d.get_state(), ref.u) < 1e-12


def test_mlp_controller_matches_oracle_decisions():
    rng = np.random.default_rng(9)
    # a network that proposes about log 1.3 with mild feature dependence
    p = (0.02 * rng.standard_normal(mlp.N_PARAMS)).astype(np.float32)
    p[-1] = math.log(1.3)
    ref, info, d = run_pair("MLP", p)
    assert (info.n_acc, info.n_rej) == (ref.n_acc, ref.n_rej)
    assert abs(info.h_next - ref.h_next) < 1e-5 * ref.h_next
    assert rel_l2(d.get_state(), ref.u) < 1e-9


def test_trace_diagnostics_match_oracle():
    from paper_1810_10197_gb300 import Dns
    shape, nu = (32, 32, 32), 0.02
    g = sp.Grid(*shape)
    uh = g.dealias(syn.random_solenoidal_hat(*shape, seed=4, k0=3.0))
    d = Dns(*shape, nu=nu)
    d.set_state(to_dev(uh), 0.0)
    d.set_trace(100, diagnostics=True)
    info = d.integrate(0.3, "BS5_ADAPTIVE", 1e-7, 1e-7, h0=0.01)
    tr = d.trace()
    assert len(tr) == info.n_acc + info.n_rej
    assert tr[-1, 4] == info.n_rhs
    u = d.get_state()
    f = sp.rhs(g, u, nu)
    assert tr[-1, 5] == pytest.approx(diag.energy(g, u), rel=1e-12)
    assert tr[-1, 6] == pytest.approx(diag.enstrophy(g, u), rel=1e-12)
    assert tr[-1, 7] == pytest.approx(diag.dissipation(g, u, f), rel=1e-10)
    # energy decays monotonically for an unforced flow
    E = tr[tr[:, 3] > 0.5, 5]
    assert np.all(np.diff(E) < 0)


def trajectories(flows):
    from paper_1810_10197_gb300 import Dns, learned
    return learned.training_set(flows, lambda shape, nu, forcing: Dns(*shape, nu=nu, forcing=forcing), to_dev)


def rt_run(shape, seed, kind, tol, T, params=None):
    """Periodic Rayleigh-Taylor (Section 3.2, the two-interface periodic setup) from rest;
    returns (final state, RHS evaluations)."""
    from paper_1810_10197_gb300 import Dns
    Y, L = syn.rayleigh_taylor_hat(*shape, seed=seed, width=0.2, amplitude=1e-2)
    d = Dns(*shape, nu=1e-3, lengths=L, boussinesq=(1e-3, 1.0))
    d.set_state(to_dev(Y), 0.0)
    if kind == "MLP":
        d.set_controller("MLP", params)
    elif kind == "PI":
        d.set_controller("PI")
    info = d.integrate(T, "BS5_ADAPTIVE", tol, tol, h0=1e-3)
    u = d.get_state()
    d.close()
    return u, info.n_rhs


def test_learned_controller_selected_on_validation_and_applied_to_held_out_rt():
    """Train candidates on PI trajectories of Taylor-Green, forced HIT and small Rayleigh-Taylor
    runs; keep the candidate that is most efficient at equal final error on a validation RT
    problem (the all-zero network, i.e. PI itself, included); apply it to a held-out RT problem
    (other seed and grid) and compare RHS evaluations at equal final error with PI and with the
    Section 2.2.1 controller over a tolerance sweep."""
    from paper_1810_10197_gb300 import learned
    flows = []
    for tol in (1e-5, 1e-6, 1e-7, 1e-8):
        for n, nu in ((32, 0.01), (32, 0.005)):
            flows.append(((n, n, n), syn.taylor_green_3d_hat(n, n, n), nu, None, tol, 2.0))
        flows.append(((32, 32, 32), syn.random_solenoidal_hat(32, 32, 32, seed=3, k0=3.0), 0.01, (2.5, 0.05),
                      tol, 1.0))
    X, T = trajectories(flows)
    Xr, Tr = [], []
    from paper_1810_10197_gb300 import Dns
    for seed in (11, 12):
        for tol in (1e-5, 1e-6, 1e-7):
            Y, L = syn.rayleigh_taylor_hat(16, 16, 32, seed=seed, width=0.2, amplitude=1e-2)
            d = Dns(16, 16, 32, nu=1e-3, lengths=L, boussinesq=(1e-3, 1.0))
            d.set_controller("PI")
            d.set_state(to_dev(Y), 0.0)
            d.set_trace(20000)
            d.integrate(3.0, "BS5_ADAPTIVE", tol, tol, h0=1e-3)
            a, b = learned.pairs_from_trace(d.trace())
            Xr.append(a)
            Tr.append(b)
            d.close()
    X, T = np.concatenate([X] + Xr), np.concatenate([T] + Tr)
    assert len(X) > 200
    tols = (1e-5, 1e-6, 1e-7)
    params, table = learned.select(X, T, lambda p, tol: rt_run((24, 24, 48), 13, "PI" if p is None else "MLP",
                                                               tol, 2.0, p), tols)
    best = max(e for _, _, e in table if e is not None)
    assert best >= 1.0        # PI is a candidate: the selection never picks a worse one
    # held-out problem: RT 32 x 32 x 64, seed 7, from rest to t = 3
    ref, _ = rt_run((32, 32, 64), 7, "I", 1e-10, 3.0)
    curves = {}
    for kind in ("I", "PI", "MLP"):
        k = "MLP" if (kind == "MLP" and params is not None) else ("PI" if kind == "MLP" else kind)
        curves[kind] = learned.sweep(lambda tol: rt_run((32, 32, 64), 7, k, tol, 3.0, params), tols, ref)
    eff_pi = learned.efficiency(curves["MLP"], curves["PI"])
    eff_i = learned.efficiency(curves["MLP"], curves["I"])
    pi_vs_i = learned.efficiency(curves["PI"], curves["I"])
    print(f"\nvalidation (RT 24x24x48, seed 13) efficiency vs PI per candidate: {table}")
    print(f"held out (RT 32x32x64, seed 7): selected network vs PI {eff_pi}, vs I {eff_i}; PI vs I {pi_vs_i}")
    print("curves (L2 error, RHS):", curves)
    # every run reaches t_end within the tolerance regime
    for c in curves.values():
        assert all(e < 1e-3 for e, _ in c)
    # the measured relation: the validation-selected controller is within 10% of PI at equal
    # error on the held-out problem (identical to PI when the selection keeps the zero network)
    assert eff_pi is not None and eff_pi >= 0.9
    if params is None:
        assert curves["MLP"] == curves["PI"]
