"""GB300 (sm_103a) Fourier pseudo-spectral Navier-Stokes right-hand side with Bogacki-Shampine
5(4) / RK4 time integration and embedded-error step control (arXiv:1810.10197).

The compute path is the C-ABI library ``libdns.so`` (CUDA kernels, declared in include/dns.h);
``paper_1810_10197_gb300.dns`` is its ctypes binding.  Build with
``python -m paper_1810_10197_gb300.build``.
"""
from .dns import (Dns, DnsError, load, declared_symbols, METHODS, SUPPORTED_N,  # noqa: F401
                  DNS_FP64, DNS_FP32_MIXED, DNS_RK4, DNS_BS5_FIXED, DNS_BS5_ADAPTIVE)
