"""Bulk copies (TMA engine) into the z pass and their bounded wait.

The z pass stages its input rows with one bulk copy per row, completing on a shared-memory
barrier.  Every wait on that barrier is bounded (about half a second): a wait that runs out
marks the step controller DNS_ERR_TIMEOUT and the CTA returns, so the context stays usable.
dns_debug_stall makes one CTA wait for 16 bytes that no copy delivers (nothing faults).
The copy modes give bit-identical results."""
import time

import numpy as np
import pytest

import synthetic as syn
from tests.gpu_helpers import lib_ready, require_gpu, to_dev, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    require_gpu()
    lib_ready()


@pytest.mark.parametrize("precision", ["fp64", "fp32x2", "fp32_mixed"])
def test_copy_modes_give_identical_results(precision):
    from paper_1810_10197_gb300 import Dns
    shape = (32, 48, 64)            # Mz = 22: rows of 22 complex values, a multiple of 16 bytes
    uh = syn.random_solenoidal_hat(*shape, seed=4, k0=3.0)
    u = to_dev(uh)
    outs = []
    for code in (0, 1, 2, 3):       # bit 0: tile variant, bit 1: element copies
        d = Dns(*shape, nu=0.02, precision=precision)
        d.set_tiles(0, code)
        f = torch.empty_like(u)
        d.rhs(u, f)
        torch.cuda.synchronize()
        outs.append(f.cpu().numpy().tobytes())
        d.close()
    assert outs[0] == outs[2] and outs[1] == outs[3]


def test_stalled_bulk_wait_reports_timeout_and_the_context_recovers():
    from paper_1810_10197_gb300 import Dns, DnsError
    shape, nu = (64, 64, 64), 0.01
    uh = syn.random_solenoidal_hat(*shape, seed=5, k0=3.0)
    d = Dns(*shape, nu=nu)
    d.set_state(to_dev(uh), 0.0)
    d.debug_stall()
    t0 = time.perf_counter()
    with pytest.raises(DnsError) as ex:
        d.step("BS5_ADAPTIVE", 0.01, 1e-6, 1e-6)
    assert ex.value.status == 7                  # DNS_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 10.0       # bounded, not a hang
    # the same context, restarted, steps normally and agrees with a fresh one bit for bit
    d.set_state(to_dev(uh), 0.0)
    info = d.step("BS5_ADAPTIVE", 0.01, 1e-6, 1e-6)
    e = Dns(*shape, nu=nu)
    e.set_state(to_dev(uh), 0.0)
    info_e = e.step("BS5_ADAPTIVE", 0.01, 1e-6, 1e-6)
    assert info.accepted == info_e.accepted == 1
    assert d.get_state().tobytes() == e.get_state().tobytes()


def test_stall_has_no_effect_with_element_copies():
    # nz = 32: Mz = 11 FP32 complex values = 88 bytes per row, not a multiple of 16: the z pass
    # copies element by element and the stall hook has nothing to stall
    from paper_1810_10197_gb300 import Dns
    shape = (32, 32, 32)
    uh = syn.random_solenoidal_hat(*shape, seed=6, k0=3.0)
    d = Dns(*shape, nu=0.01, precision="fp32_mixed")
    d.set_state(to_dev(uh), 0.0)
    d.debug_stall()
    info = d.step("BS5_ADAPTIVE", 0.01, 1e-5, 1e-5)
    assert info.accepted in (0, 1) and np.isfinite(info.err)
