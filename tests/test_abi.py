"""CPU checks of the C-ABI library: it builds, loads, and exports every symbol dns.h declares.

No compute call is made here (there is no GPU in the CPU suite); only argument checks that
return before touching CUDA are exercised.
"""
import ctypes as C
import os
import re
import shutil

import pytest

import paper_1810_10197_gb300 as pkg
from paper_1810_10197_gb300 import build, dns


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists(dns.LIB_PATH):
        pytest.skip("no nvcc and no prebuilt libdns.so")
    build.build()
    return dns.load()


def test_header_declares_the_boundary():
    names = dns.declared_symbols()
    for required in ("dns_create", "dns_destroy", "dns_set_state", "dns_get_state", "dns_rhs",
                     "dns_step", "dns_integrate", "dns_diagnostics", "dns_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in dns.declared_symbols():
        assert hasattr(lib, name), name
    # and the binding covers them all
    assert set(dns.declared_symbols()) <= set(dns._SIGS)


def test_exports_are_c_abi_only(lib):
    out = os.popen(f"nm -D --defined-only {dns.LIB_PATH}").read()
    exported = set(re.findall(r" T (\w+)", out))
    # only the C ABI leaves the library: every other symbol is hidden
    assert exported == set(dns.declared_symbols())


def test_argument_checks_before_cuda(lib):
    h = C.c_void_p()
    # unsupported size and bad config are rejected before any CUDA call
    assert lib.dns_create(10, 16, 16, 0.01, None, 0, C.byref(h)) == 9        # DNS_ERR_UNSUPPORTED
    assert lib.dns_create(16, 16, 16, -1.0, None, 0, C.byref(h)) == 1        # DNS_ERR_ARG
    assert lib.dns_create(16, 16, 16, 0.01, None, 7, C.byref(h)) == 1        # bad precision
    assert lib.dns_create_ex(None, C.byref(h)) == 1
    assert lib.dns_step(None, 2, 0.1, 1e-6, 1e-6, 1.0, None) == 1
    assert lib.dns_rhs(None, None, None) == 1
    assert lib.dns_query(None, None, None) == 1


def test_build_flags_target_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert pkg.SUPPORTED_N == (8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768)


def test_checkpoint_crc32_is_zlib_crc32(lib):
    # the checkpoint trailer is the standard CRC-32 (reflected 0xEDB88320), pinned to zlib
    import zlib
    rng = __import__("numpy").random.default_rng(3)
    data = rng.integers(0, 256, 100003, dtype="uint8").tobytes()
    assert dns.dns_crc32(b"") == 0
    assert dns.dns_crc32(b"123456789") == 0xCBF43926        # the published check value
    assert dns.dns_crc32(data) == zlib.crc32(data)
    # continuation over split buffers equals one pass
    assert dns.dns_crc32(data[5000:], dns.dns_crc32(data[:5000])) == zlib.crc32(data)


def test_checkpoint_calls_check_arguments_before_cuda(lib):
    assert lib.dns_save(None, b"x") == 1
    assert lib.dns_load(None, b"x") == 1
