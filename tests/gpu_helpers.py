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


def err_tolerance(h, ks, e, tab, eps_rhs=1e-13):
    """Relative tolerance for the embedded error norm.

    e = h sum_j (b_j - bhat_j) k_j cancels heavily: a relative rounding error eps_rhs in each
    k_j becomes eps_rhs * h sum_j |b_j - bhat_j| max|k_j| / max|e| in e (and in err).
    """
    num = h * sum(abs(float(b - bh)) * float(np.max(np.abs(k)))
                  for b, bh, k in zip(tab.b, tab.bhat, ks))
    return eps_rhs * num / float(np.max(np.abs(e)))
