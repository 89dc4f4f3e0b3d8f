"""Pins for the learned-controller reference (oracle/mlp.py) and the PI controller."""
import math
import os

import numpy as np
import pytest

from oracle import mlp, rk

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_parameter_count():
    assert mlp.N_PARAMS == 64 * 16 + 64 + 64 * 64 + 64 + 64 + 1 == 5313


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    p = mlp.init_params(1) + 0.01 * rng.standard_normal(mlp.N_PARAMS)
    X = rng.standard_normal((37, 16))
    t = rng.standard_normal(37)
    L, g = mlp.loss_and_grad(p, X, t)
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = 1e-6
        num = (mlp.loss_and_grad(p + e, X, t)[0] - mlp.loss_and_grad(p - e, X, t)[0]) / 2e-6
        assert abs(num - g[i]) <= 1e-7 * max(1.0, abs(g[i])), (i, num, g[i])


def test_forward_is_the_stated_network():
    # a network whose only path is x0 -> unit 0 -> unit 0 -> output computes 3*relu(2*relu(x0))+1
    p = np.zeros(mlp.N_PARAMS)
    W1, b1, W2, b2, w3, b3 = (None,) * 6
    p[0] = 1.0                                   # W1[0][0]
    o = 64 * 16 + 64
    p[o + 0] = 2.0                               # W2[0][0]
    o += 64 * 64 + 64
    p[o + 0] = 3.0                               # w3[0]
    p[-1] = 1.0                                  # b3
    X = np.zeros((3, 16))
    X[:, 0] = [-1.0, 0.5, 2.0]
    y, _ = mlp.forward(p, X)
    assert np.allclose(y, [1.0, 4.0, 13.0])


def test_bf16_rounding():
    vals = np.array([1.0, 1.00390625, 1.001953125, 3.14159265, -2.5e-3, 0.0])
    r = mlp.round_bf16(vals)
    # bf16 keeps 8 significant bits: 1 + 2^-8 is representable? no: spacing at 1 is 2^-7
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0
    assert abs(r[3] - 3.140625) < 1e-12
    assert r[5] == 0.0
    assert np.all(np.abs(r - vals) <= np.abs(vals) * 2 ** -8 + 1e-30)


def test_dataset_targets_are_hindsight_steps():
    # history: accepted steps with known errors; target = log(h_{n+1} (e*/err_{n+1})^(1/5) / h_n)
    # with e* the PI factor's fixed point: 0.8 e^(-0.14) e^(0.08) = 1, e* = 0.8^(1/0.06)
    estar = math.exp(math.log(0.8) / 0.06)
    assert abs(estar - 0.024257) < 1e-6 and abs(mlp.E_TARGET - estar) < 1e-14
    assert abs(rk.pi_factor(estar, estar, False) - 1.0) < 1e-13
    steps = [(0, 0.1, 0.5, True), (0.1, 0.1, 0.5, True), (0.2, 0.1, 0.25, True), (0.3, 0.2, 2.0, False),
             (0.3, 0.12, 0.4, True), (0.42, 0.15, estar, True)]
    X, T = mlp.dataset_from_history(steps)
    assert X.shape == (1, 16)
    # n = 3 (4th accepted: h=0.12, err 0.4), next accepted h=0.15 with err = e* -> h* = 0.15;
    # the PI factor at n is 0.8 * 0.4^(-0.14) * 0.25^(0.08): err_prev is the accepted step
    # before it (0.25), not the rejected attempt (2.0).  Worked by hand: 0.4^-0.14 = 1.136872,
    # 0.25^0.08 = 0.895025, factor 0.814023, target log(1.25) - log(0.814023) = 0.428910
    assert abs(T[0] - (math.log(0.15 / 0.12) - math.log(0.8 * 0.4 ** -0.14 * 0.25 ** 0.08))) < 1e-12
    assert abs(T[0] - 0.428910) < 2e-6
    # a next error 32x the target halves the hindsight step: the target drops by log 2
    steps[-1] = (0.42, 0.15, 32 * estar, True)
    X2, T2 = mlp.dataset_from_history(steps)
    assert abs(T2[0] - (T[0] - math.log(2.0))) < 1e-12
    # features: newest accepted err 0.4 with 1 rejection before it
    assert abs(X[0, 0] - math.log10(0.4)) < 1e-12 and X[0, 2] == 1.0 and X[0, 1] == 0.0


def test_pi_factor_hand_worked():
    with open(os.path.join(GOLDEN, "pi_controller_cases.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    for err, errp, after, fac in rows:
        got = rk.pi_factor(float(err), float(errp), bool(int(after)))
        assert abs(got - float(fac)) < 1e-13, (err, errp, after, got, fac)


def test_learned_proposal_is_a_bounded_correction_of_the_pi_controller():
    hist = [(0.1, 0.05, 0), (0.2, 0.04, 1), (0.3, 0.04, 0), (0.3, 0.03, 0)]
    fac_pi = rk.pi_factor(0.1, 0.2, False)                             # 0.8 0.1^-0.14 0.2^0.08
    assert abs(fac_pi - 0.8 * 1.380384 * 0.879189) < 1e-6              # worked by hand
    p = np.zeros(mlp.N_PARAMS)
    assert abs(mlp.propose_factor(p, hist, 0.2) - fac_pi) < 1e-12      # y = 0: plain PI controller
    p[-1] = 10.0                                                       # y clamped to log 1.5
    assert abs(mlp.propose_factor(p, hist, 0.2) - min(2.0, 1.5 * fac_pi)) < 1e-12
    p[-1] = -10.0
    assert abs(mlp.propose_factor(p, hist, 0.2) - fac_pi / 1.5) < 1e-12
    p[-1] = 10.0                                                       # the upper bound 2 applies
    assert mlp.propose_factor(p, [(1e-6,) + hist[0][1:]] + hist[1:], 1e-6) == 2.0


def test_zero_network_integrates_like_the_pi_controller():
    # y = 0 makes the learned controller the PI controller it corrects: the same accept/reject
    # sequence and step sizes on a stiff-ish linear system u' = -diag(lam) u whose error
    # estimates vary from step to step.  The factors differ in rounding only (exp of a sum of
    # logs against a product of powers, ~1e-16), which the embedded estimate, a cancellation,
    # amplifies over the run: measured 2e-11 relative in h after 73 attempts; bound 1e-9
    lam = np.array([1.0, 7.0, 40.0])

    def f(u):
        return -lam[:, None] * u

    u0 = np.ones((3, 4))
    p = np.zeros(mlp.N_PARAMS)
    a = rk.integrate(f, u0, 0.0, 3.0, "BS5_ADAPTIVE", 0.3, 1e-7, 1e-7, controller="PI")
    b = rk.integrate(f, u0, 0.0, 3.0, "BS5_ADAPTIVE", 0.3, 1e-7, 1e-7, controller=("MLP", p))
    c = rk.integrate(f, u0, 0.0, 3.0, "BS5_ADAPTIVE", 0.3, 1e-7, 1e-7, controller="I")
    assert a.n_rej > 0 and a.n_acc > 10
    assert (a.n_acc, a.n_rej) == (b.n_acc, b.n_rej)
    for (ta, ha, ea, oka), (tb, hb, eb, okb) in zip(a.history, b.history):
        assert oka == okb and hb == pytest.approx(ha, rel=1e-9)
    # and it is not the Section 2.2.1 controller's trajectory
    assert [h for _, h, _, _ in c.history] != pytest.approx([h for _, h, _, _ in a.history], rel=1e-6)
