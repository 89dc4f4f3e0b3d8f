"""Shared helpers for the GPU parity tests (loaded by tests marked gpu)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")


def lib_ready():
    from paper_1810_10197_gb300 import build, dns
    build.build()
    return dns.load()


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def rel_l2(a, b):
    nb = np.linalg.norm(np.ravel(b))
    return np.linalg.norm(np.ravel(a - b)) / (nb if nb > 0 else 1.0)


def rel_max(a, b):
    mb = np.max(np.abs(b))
    return np.max(np.abs(a - b)) / (mb if mb > 0 else 1.0)


def err_tolerance(h, ks, e, tab, u_old, u_new, atol, rtol, eps_rhs=1e-13):
    """Relative tolerance for the embedded error norm err = max_c sqrt(mean (|e|/sc)^2).

    The CUDA and oracle right-hand sides agree to eps_rhs relative to each field's largest
    entry, so every mode of e = h sum_j (b_j - bhat_j) k_j carries an absolute error up to
    de = eps_rhs h sum_j |b_j - bhat_j| max|k_j|, independent of the mode.  Linearising
    err^2 = mean(|e|^2/sc^2) gives d(err)/err <= sum |e| de / sc^2 / sum |e|^2 / sc^2 for the
    component that attains the maximum (the bound is taken over all components).
    """
    de = eps_rhs * h * sum(abs(float(b - bh)) * float(np.max(np.abs(k)))
                           for b, bh, k in zip(tab.b, tab.bhat, ks))
    sc = atol + rtol * np.maximum(np.abs(u_old), np.abs(u_new))
    ae = np.abs(e)
    # modes with e = 0 contribute nothing to the norm (also where sc = 0, atol = 0)
    live = ae > 0
    isc2 = np.where(live, 1.0 / np.where(live, sc, 1.0) ** 2, 0.0)
    rel = 0.0
    for c in range(e.shape[0]):
        num = float(np.sum(ae[c] * de * isc2[c]))
        den = float(np.sum(ae[c] ** 2 * isc2[c]))
        if den > 0:
            rel = max(rel, num / den)
    return rel + 1e-15
