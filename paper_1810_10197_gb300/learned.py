"""Training pipeline for the learned step-size proposal (DNS_CTRL_MLP).

Trajectories come from the device attempt trace (dns_set_trace / dns_trace) of runs with the
PI controller, the base the learned proposal corrects; the training pairs are built on the
host (a few thousand rows) and the network is trained on the GPU by the library's own
kernels (dns_mlp_train).

Features at accepted step n (newest first, i = 0..3, h_0 = h_n):
    [log10 err_i, log(h_i / h_0), rejections just before step i, log(h_i / h_{i+1})]
Target: log(h*_n / h_n) - log(0.8 err_n^(-0.7/5) e_n^(0.4/5)) with
h*_n = h_{n+1} (E_TARGET / err_{n+1})^(1/5), n+1 the next accepted step and e_n the error of
the last earlier accepted step with a positive error (1 if none): the step that in hindsight
gives the error the PI controller settles at, E_TARGET = 0.8^(1/(0.7/5 - 0.4/5)) (the fixed
point of its factor at constant error), relative to the PI proposal.  The network learns a
bounded correction of PI's prediction, not of the error level PI keeps.
"""
from __future__ import annotations

import math

import numpy as np

from . import dns as _dns

E_TARGET = 0.8 ** (1.0 / (0.7 / 5.0 - 0.4 / 5.0))


def _features(hist):
    h0 = hist[0][1]
    out = []
    for i in range(4):
        err, h, rej = hist[i]
        hp = hist[i + 1][1] if i + 1 < len(hist) else h
        out += [math.log10(max(err, 1e-300)), math.log(h / h0), float(rej), math.log(h / hp)]
    return out


def pairs_from_trace(trace: np.ndarray):
    """(X[n,16], T[n]) from an attempt trace (columns t, h, err, accepted, ...)."""
    acc, eprev, rej, e_last = [], [], 0, 1.0
    for row in trace:
        h, err, ok = float(row[1]), float(row[2]), row[3] > 0.5
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
        err1, h1, _ = acc[n + 1]
        errn = acc[n][0]
        if not (err1 > 0 and math.isfinite(err1) and errn > 0):
            continue
        hist = [acc[n - i] for i in range(min(5, n + 1))]
        X.append(_features(hist))
        T.append(math.log(h1 * (E_TARGET / err1) ** 0.2 / acc[n][1])
                 - math.log(0.8 * errn ** -0.14 * eprev[n] ** 0.08))
    return np.asarray(X, dtype=np.float32).reshape(-1, 16), np.asarray(T, dtype=np.float32)


def init_params(seed=0):
    """He-style initial parameters (float32), layout of dns.h DNS_MLP_PARAMS."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((64, 16)) * math.sqrt(2.0 / 16)
    W2 = rng.standard_normal((64, 64)) * math.sqrt(2.0 / 64)
    w3 = rng.standard_normal(64) * math.sqrt(1.0 / 64)
    p = np.concatenate([W1.ravel(), np.zeros(64), W2.ravel(), np.zeros(64), w3, [0.0]])
    return p.astype(np.float32)


def train(X: np.ndarray, T: np.ndarray, steps=3000, batch=128, lr=2e-3, seed=0):
    """Train on the GPU; returns (params as a device tensor, batch-loss history)."""
    import torch
    dev = torch.device("cuda")
    x = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(dev)
    t = torch.from_numpy(np.ascontiguousarray(T, dtype=np.float32)).to(dev)
    p = torch.from_numpy(init_params(seed)).to(dev)
    hist = torch.zeros(max(steps, 1), dtype=torch.float32, device=dev)
    st = _dns.dns_mlp_train(p, x, t, steps, batch=min(batch, 128), lr=lr, seed=seed, loss_hist=hist,
                            stream=torch.cuda.current_stream())
    if st != 0:
        raise _dns.DnsError(st, "dns_mlp_train")
    torch.cuda.synchronize()
    return p, hist.cpu().numpy()


def training_set(flows, make_dns, to_dev):
    """Pairs from runs of the PI controller: flows = [(shape, uhat, nu, forcing, tol, T)]."""
    Xs, Ts = [], []
    for (shape, uh, nu, forcing, tol, T) in flows:
        d = make_dns(shape, nu, forcing)
        d.set_controller("PI")
        d.set_state(to_dev(uh), 0.0)
        d.set_trace(20000)
        d.integrate(T, "BS5_ADAPTIVE", tol, tol, h0=1e-3)
        X, Tt = pairs_from_trace(d.trace())
        Xs.append(X)
        Ts.append(Tt)
        d.close()
    return np.concatenate(Xs), np.concatenate(Ts)


# ---- model selection on a validation problem ----------------------------------------------

def at_error(base, e):
    """log-log interpolation of the RHS count of an error-versus-cost curve
    base = [(l2_error, rhs_evals), ...] at error e (None outside its range)."""
    pts = sorted((err, r) for err, r in base if err > 0)
    for (e0, r0), (e1, r1) in zip(pts, pts[1:]):
        if e0 <= e <= e1:
            w = (math.log(e) - math.log(e0)) / (math.log(e1) - math.log(e0)) if e1 > e0 else 0.0
            return math.exp(math.log(r0) + w * (math.log(r1) - math.log(r0)))
    return None


def efficiency(curve, base):
    """Geometric mean, over the points of `curve` inside `base`'s error range, of base's RHS
    count at the same final error divided by curve's: above 1, `curve` reaches the same error
    with fewer right-hand sides.  None if no point is comparable."""
    r = [at_error(base, e) / n for e, n in curve if e > 0 and at_error(base, e) is not None]
    return math.exp(sum(math.log(x) for x in r) / len(r)) if r else None


def sweep(run, tols, reference):
    """[(final L2 error against `reference`, RHS evaluations)] of run(tol) -> (state, n_rhs)."""
    nrm = float(np.linalg.norm(reference))
    out = []
    for tol in tols:
        u, n = run(tol)
        out.append((float(np.linalg.norm(u - reference)) / nrm, int(n)))
    return out


def select(X, T, run_validation, tols, steps_grid=(150, 500, 1500, 3000), seeds=(0, 1), lr=2e-3):
    """Train candidate networks (every step count and seed of the grids) and keep the one that
    reaches a given final error with the fewest right-hand sides on a validation problem,
    against the PI controller (the all-zero network, which is exactly PI, is a candidate too).

    run_validation(params or None, tol) -> (final state, n_rhs); params None runs PI, and the
    validation reference is run_validation's own tol-1e-10 PI run.  Returns (params as a
    device tensor or None, table of (steps, seed, efficiency vs PI))."""
    import torch
    ref, _ = run_validation(None, 1e-10)
    base = sweep(lambda tol: run_validation(None, tol), tols, ref)
    best, best_eff, table = None, 1.0, [("PI", None, 1.0)]
    for steps in steps_grid:
        for seed in seeds:
            p, _ = train(X, T, steps=steps, lr=lr, seed=seed)
            curve = sweep(lambda tol: run_validation(p, tol), tols, ref)
            eff = efficiency(curve, base)
            table.append((steps, seed, eff))
            if eff is not None and eff > best_eff:
                best, best_eff = p, eff
            torch.cuda.synchronize()
    return best, table
