"""Scratch poisoning (dns_debug_poison): with the pass scratch buffers filled with NaN bytes
before every right-hand side, every form and layout must give results identical, bit for bit,
to a run without it -- no pass reads scratch that an earlier pass of the same evaluation did
not write.  Covers the odd line lengths (radix 3), non-cubic grids, the 3/2 rule, the
Boussinesq form and the integrate graph."""
import numpy as np
import pytest

import synthetic as syn
from tests.gpu_helpers import lib_ready, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    require_gpu()
    lib_ready()


CASES = [((16, 16, 16), "fp64", {}), ((12, 24, 48), "fp64", {}), ((24, 12, 8), "fp32_mixed", {}),
         ((32, 48, 64), "fp32_mixed", {}), ((32, 64, 48), "fp32x2", {}), ((48, 32, 32), "fp32x2", {}),
         ((32, 32, 32), "fp64", {"dealias": "3/2"}), ((32, 32, 32), "fp32x2", {"dealias": "3/2"}),
         ((16, 16, 32), "fp64", {"boussinesq": (0.01, 1.0)}),
         ((16, 16, 32), "fp32_mixed", {"boussinesq": (0.01, 1.0)}),
         ((32, 32, 32), "fp32", {"dealias": "3/2"}), ((16, 16, 32), "fp32", {"boussinesq": (0.01, 1.0)})]


@pytest.mark.parametrize("shape,precision,kw", CASES)
def test_rhs_identical_with_poisoned_scratch(shape, precision, kw):
    from paper_1810_10197_gb300 import Dns
    nc = 4 if "boussinesq" in kw else 3
    uh = syn.random_solenoidal_hat(*shape, seed=sum(shape), k0=3.0)
    if nc == 4:
        uh = np.concatenate([uh, syn.random_complex_hat(*shape, seed=5, ncomp=1)])
    d = Dns(*shape, nu=0.02, precision=precision, **kw)
    u = to_dev(uh)
    f0, f1 = torch.empty_like(u), torch.empty_like(u)
    d.rhs(u, f0)
    d.debug_poison(True)
    d.rhs(u, f1)
    torch.cuda.synchronize()
    a, b = f0.cpu().numpy(), f1.cpu().numpy()
    assert np.all(np.isfinite(b))
    assert a.tobytes() == b.tobytes()
    d.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32x2", "fp32"])
def test_integrate_identical_with_poisoned_scratch(precision):
    from paper_1810_10197_gb300 import Dns
    shape = (32, 32, 32)
    uh = syn.random_solenoidal_hat(*shape, seed=3, k0=3.0)
    out = []
    for poison in (False, True):
        d = Dns(*shape, nu=0.01, precision=precision)
        d.debug_poison(poison)
        d.set_state(to_dev(uh), 0.0)
        info = d.integrate(0.1, "BS5_ADAPTIVE", 1e-7, 1e-7, h0=0.01)
        out.append((info.n_acc, info.n_rej, d.get_state().tobytes()))
        d.close()
    assert out[0] == out[1]
