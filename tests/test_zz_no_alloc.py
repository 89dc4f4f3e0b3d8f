"""dns_rhs_noalloc: the allocation-free right-hand side for small grids.

Some callers cannot call cudaMalloc (a host program that hands out all device memory
through its own pool, or a latency-critical path where cudaMalloc/cudaFree would
synchronise the device).  dns_rhs_noalloc serves them with a static device work space;
this test checks, through the C ABI, that two calls in a row give the same result as the
context-based dns_rhs and as the FP64 oracle, within the FP64 right-hand-side tolerance of
the other tests, and that sizes beyond its 32^3 limit are refused.  It runs alone or after
the other tests.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle import spectral as sp
from tests.gpu_helpers import lib_ready, rel_max, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-13   # same bound as the dns_rhs parity tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    require_gpu()
    lib_ready()


def rhs_with_context(shape, uh, nu):
    from paper_1810_10197_gb300 import Dns
    d = Dns(*shape, nu=nu)
    u = to_dev(uh)
    f = torch.empty_like(u)
    d.rhs(u, f)
    torch.cuda.synchronize()
    out = f.cpu().numpy()
    d.close()
    return out


@pytest.mark.parametrize("shape", [(32, 32, 32), (16, 24, 8)])
def test_noalloc_matches_dns_rhs_on_two_calls_in_a_row(shape):
    from paper_1810_10197_gb300.dns import dns_rhs_noalloc
    nu = 0.011
    fields = [syn.random_solenoidal_hat(*shape, seed=21, k0=3.0),
              syn.random_complex_hat(*shape, seed=22)]
    outs = []
    for uh in fields:
        u = to_dev(uh)
        f = torch.full_like(u, complex(np.nan, np.nan))
        st = dns_rhs_noalloc(*shape, nu, u, f)
        assert st == 0
        torch.cuda.synchronize()
        outs.append(f.cpu().numpy())
    g = sp.Grid(*shape)
    for uh, got in zip(fields, outs):
        ref = rhs_with_context(shape, uh, nu)
        assert rel_max(got, ref) < FP64_TOL
        # and directly against the FP64 oracle's right-hand side (Eq. ufdef, 2/3 rule)
        assert rel_max(got, sp.rhs(g, g.dealias(uh), nu)) < FP64_TOL


def test_noalloc_refuses_sizes_beyond_its_limit():
    from paper_1810_10197_gb300.dns import dns_rhs_noalloc
    u = torch.zeros((3, 64, 64, 33), dtype=torch.complex128, device="cuda")
    f = torch.empty_like(u)
    assert dns_rhs_noalloc(64, 64, 64, 0.01, u, f) == 9        # DNS_ERR_UNSUPPORTED
    u = torch.zeros((3, 32, 32, 17), dtype=torch.complex128, device="cuda")
    f = torch.empty_like(u)
    assert dns_rhs_noalloc(32, 32, 32, -1.0, u, f) == 1        # DNS_ERR_ARG
    # the binding refuses buffers the kernels would overrun before calling the library
    with pytest.raises(ValueError):
        dns_rhs_noalloc(32, 32, 32, 0.01, u.cpu(), f)                        # host memory
    with pytest.raises(ValueError):
        dns_rhs_noalloc(32, 32, 32, 0.01, u.to(torch.complex64), f)          # wrong dtype
    with pytest.raises(ValueError):
        dns_rhs_noalloc(32, 32, 32, 0.01, u[:2], f)                          # too short
