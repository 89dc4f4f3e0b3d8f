"""Learned step-size proposal: a 16-64-64-1 multilayer perceptron, FP64 reference.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper's step-size controller is
the elementary one of Section 2.2.1 and it names better controllers as future work
(Section 4); this module is the reference for the learned variant built on the PI controller
(factor 0.8 err^(-0.7/5) err_prev^(0.4/5), err_prev the error of the previous accepted step).
The network proposes a bounded correction of the PI factor from the recent accepted-step
history: h_next = h min(2, max(0.01, 0.8 err^(-0.7/5) err_prev^(0.4/5) exp(clamp(y, +-log 1.5)))).
An uncertain network (y near 0) behaves like the PI controller, which is also the fallback
(the first accepted steps, a non-finite output); the embedded error estimate still accepts or
rejects every step, and a rejected attempt takes the Section 2.2.1 factor.

Parameter vector (float, length N_PARAMS), in this order:
  W1[64][16], b1[64], W2[64][64], b2[64], w3[64], b3[1]
Forward:  a1 = relu(W1 x + b1), a2 = relu(W2 a1 + b2), y = w3 . a2 + b3
Loss:     L = mean_b (y_b - t_b)^2

Features of the history (4 most recent accepted steps, newest first, i = 0..3), each
  [log10 err_i, log(h_i / h_0), rejections just before step i, log(h_i / h_{i+1})]
with h_0 the newest accepted step (the last feature of i = 3 uses the step before it, or 0).
Target for training at accepted step n: log(h*_n / h_n) - log(0.8 err_n^(-0.7/5) e_n^(0.4/5)),
with e_n the error of the last accepted step before n with a positive error (1 if none),
h*_n = h_{n+1} (E_TARGET/err_{n+1})^(1/5) and n+1 the next accepted step -- the step that, in
hindsight, would have produced the error the PI controller settles at (error ~ h^5 for the
4th-order embedded estimate), relative to what the PI controller proposed.  That level is the
fixed point of the PI factor at constant error, 0.8 e^(-0.7/5 + 0.4/5) = 1, so
E_TARGET = 0.8^(1/0.06) = 0.0243: the network corrects the PI controller's prediction of the
next error, not the error level it keeps.
"""
from __future__ import annotations

import math

import numpy as np

NIN, NH, NOUT = 16, 64, 1
N_PARAMS = NH * NIN + NH + NH * NH + NH + NH + 1
LOG_DMIN, LOG_DMAX = math.log(0.01), math.log(2.0)
LOG_CORR = math.log(1.5)      # bound of the learned correction
PI_ALPHA, PI_BETA = 0.7 / 5.0, 0.4 / 5.0
E_TARGET = 0.8 ** (1.0 / (PI_ALPHA - PI_BETA))   # fixed point of the PI factor


def log_pi_factor(err, err_prev):
    """log of the unclamped PI factor 0.8 err^(-alpha) err_prev^beta (err, err_prev > 0)."""
    return math.log(0.8) - PI_ALPHA * math.log(err) + PI_BETA * math.log(err_prev)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + NH * NIN].reshape(NH, NIN); o += NH * NIN
    b1 = p[o:o + NH]; o += NH
    W2 = p[o:o + NH * NH].reshape(NH, NH); o += NH * NH
    b2 = p[o:o + NH]; o += NH
    w3 = p[o:o + NH]; o += NH
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def round_bf16(p):
    """Round float values to bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(p, dtype=np.float32).copy()
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(p, X):
    """y for a batch X[B][16]; also returns the activations for backward."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    z1 = X @ W1.T + b1
    a1 = np.maximum(z1, 0.0)
    z2 = a1 @ W2.T + b2
    a2 = np.maximum(z2, 0.0)
    y = a2 @ w3 + b3
    return y, (X, z1, a1, z2, a2)


def loss_and_grad(p, X, t):
    """Mean squared error and its gradient with respect to the parameter vector."""
    W1, b1, W2, b2, w3, b3 = unpack(p)
    y, (X, z1, a1, z2, a2) = forward(p, X)
    B = X.shape[0]
    r = y - t
    L = float(np.mean(r * r))
    dy = 2.0 * r / B
    dw3 = a2.T @ dy
    db3 = np.sum(dy)
    da2 = np.outer(dy, w3) * (z2 > 0)
    dW2 = da2.T @ a1
    db2 = np.sum(da2, axis=0)
    da1 = (da2 @ W2) * (z1 > 0)
    dW1 = da1.T @ X
    db1 = np.sum(da1, axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])
    return L, g


def init_params(seed=0):
    """He-style initial weights from a seeded generator (biases zero)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((NH, NIN)) * math.sqrt(2.0 / NIN)
    W2 = rng.standard_normal((NH, NH)) * math.sqrt(2.0 / NH)
    w3 = rng.standard_normal(NH) * math.sqrt(1.0 / NH)
    return np.concatenate([W1.ravel(), np.zeros(NH), W2.ravel(), np.zeros(NH), w3, [0.0]])


def features(hist):
    """16 features from the 4 newest accepted steps, hist = [(err, h, rejects_before), ...]
    newest first (len >= 4)."""
    h0 = hist[0][1]
    out = []
    for i in range(4):
        err, h, rej = hist[i]
        hprev = hist[i + 1][1] if i + 1 < len(hist) else h
        out += [math.log10(max(err, 1e-300)), math.log(h / h0), float(rej), math.log(h / hprev)]
    return np.array(out)


def dataset_from_history(steps):
    """Training pairs from one run's attempt history [(t, h, err, accepted), ...]."""
    acc = []            # (err, h, rejections before it)
    eprev = []          # error of the last earlier accepted step with err > 0 (1 if none)
    rej = 0
    e_last = 1.0
    for (_, h, err, ok) in steps:
        if ok:
            acc.append((err, h, rej))
            eprev.append(e_last)
            if err > 0:
                e_last = err
            rej = 0
        else:
            rej += 1
    X, T = [], []
    for n in range(3, len(acc) - 1):
        hist = [acc[n - i] for i in range(min(5, n + 1))]
        err1, h1, _ = acc[n + 1]
        errn = acc[n][0]
        if not (err1 > 0 and math.isfinite(err1) and errn > 0):
            continue
        hstar = h1 * (E_TARGET / err1) ** 0.2
        X.append(features(hist))
        T.append(math.log(hstar / acc[n][1]) - log_pi_factor(errn, eprev[n]))
    return np.array(X).reshape(-1, NIN), np.array(T)


def propose_factor(p, hist, err_prev):
    """Step factor fac_PI exp(clamp(y, +-log 1.5)) clamped to [dmin, dmax] (weights rounded to
    bf16); hist[0] is the step just accepted, err_prev the error of the accepted step before
    it (1 if none).  None if y is not finite."""
    y, _ = forward(round_bf16(p), features(hist)[None, :])
    y = float(y[0])
    err = hist[0][0]
    if not math.isfinite(y) or not err > 0:
        return None
    lf = log_pi_factor(err, err_prev) + min(LOG_CORR, max(-LOG_CORR, y))
    return math.exp(min(LOG_DMAX, max(LOG_DMIN, lf)))
