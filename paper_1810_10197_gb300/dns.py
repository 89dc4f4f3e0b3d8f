"""ctypes binding for libdns (include/dns.h).  Argument marshalling only: every step of the
right-hand side and of the time integration runs in the library's CUDA kernels.

Module-level functions carry the C names (``dns_create``, ``dns_rhs``, ...).  The ``Dns``
class wraps one context.  torch tensors are passed by ``data_ptr()``; numpy arrays (host) by
their buffer address.  Spectral fields are complex128 arrays of shape (3, nx, ny, nz//2+1).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdns.so")
HEADER_PATH = os.path.join(os.path.dirname(_PKG), "include", "dns.h")

DNS_OK = 0
DNS_ERR_ARG = 1
STATUS_NAMES = {0: "DNS_OK", 1: "DNS_ERR_ARG", 2: "DNS_ERR_CUDA", 3: "DNS_ERR_OOM",
                4: "DNS_ERR_NONFINITE", 5: "DNS_ERR_STEP_UNDERFLOW", 6: "DNS_ERR_MAX_REJECTS",
                7: "DNS_ERR_TIMEOUT", 8: "DNS_ERR_STATE", 9: "DNS_ERR_UNSUPPORTED"}
DNS_RK4, DNS_BS5_FIXED, DNS_BS5_ADAPTIVE, DNS_DP5_FIXED, DNS_DP5_ADAPTIVE = 0, 1, 2, 3, 4
METHODS = {"RK4": DNS_RK4, "BS5_FIXED": DNS_BS5_FIXED, "BS5_ADAPTIVE": DNS_BS5_ADAPTIVE,
           "DP5_FIXED": DNS_DP5_FIXED, "DP5_ADAPTIVE": DNS_DP5_ADAPTIVE}
DNS_FP64, DNS_FP32_MIXED, DNS_FP32X2, DNS_FP32 = 0, 1, 2, 3
PRECISIONS = {"fp64": DNS_FP64, "fp32_mixed": DNS_FP32_MIXED, "fp32x2": DNS_FP32X2, "fp32": DNS_FP32}
SUPPORTED_N = (8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768)


class dns_forcing(C.Structure):
    _fields_ = [("kind", C.c_int), ("kf", C.c_double), ("power", C.c_double)]


class dns_config(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("lx", C.c_double), ("ly", C.c_double), ("lz", C.c_double),
                ("nu", C.c_double), ("precision", C.c_int), ("forcing", dns_forcing),
                ("dealias", C.c_int)]


class dns_step_info(C.Structure):
    _fields_ = [("accepted", C.c_int), ("status", C.c_int), ("err", C.c_double),
                ("h_used", C.c_double), ("h_next", C.c_double), ("t", C.c_double),
                ("n_rhs", C.c_longlong), ("n_acc", C.c_longlong), ("n_rej", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class DnsError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")


_lib = None

_SIGS = {
    "dns_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(dns_forcing), C.c_int,
                             C.POINTER(C.c_void_p)]),
    "dns_create_ex": (C.c_int, [C.POINTER(dns_config), C.POINTER(C.c_void_p)]),
    "dns_create_boussinesq": (C.c_int, [C.POINTER(dns_config), C.c_double, C.c_double,
                                        C.POINTER(C.c_void_p)]),
    "dns_destroy": (None, [C.c_void_p]),
    "dns_last_error": (C.c_char_p, [C.c_void_p]),
    "dns_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dns_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_double]),
    "dns_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "dns_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dns_step": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                           C.POINTER(dns_step_info)]),
    "dns_integrate": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_double, C.c_double, C.c_double,
                                C.c_int, C.POINTER(dns_step_info)]),
    "dns_enqueue_attempts": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_double,
                                       C.c_double, C.c_double]),
    "dns_get_info": (C.c_int, [C.c_void_p, C.POINTER(dns_step_info)]),
    "dns_diagnostics": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                  C.POINTER(C.c_double)]),
    "dns_profile_enable": (C.c_int, [C.c_void_p, C.c_int]),
    "dns_profile_count": (C.c_int, [C.c_void_p]),
    "dns_profile_get": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_longlong),
                                  C.POINTER(C.c_double)]),
    "dns_query": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_size_t)]),
    "dns_rhs_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p,
                                  C.c_void_p]),
    "dns_set_trace": (C.c_int, [C.c_void_p, C.c_longlong, C.c_int]),
    "dns_trace": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.POINTER(C.c_longlong)]),
    "dns_set_controller": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "dns_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "dns_mlp_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                    C.c_void_p, C.c_void_p]),
    "dns_mlp_train": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                C.c_float, C.c_uint, C.c_void_p, C.c_void_p]),
}
_SIGS.update({
    "dns_spectrum": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "dns_autotune": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    "dns_set_tiles": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "dns_create_batch": (C.c_int, [C.c_int, C.POINTER(dns_config), C.POINTER(C.c_void_p)]),
    "dns_destroy_batch": (None, [C.c_void_p]),
    "dns_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "dns_batch_context": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p)]),
    "dns_integrate_batch": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(dns_step_info)]),
    "dns_debug_poison": (C.c_int, [C.c_void_p, C.c_int]),
    "dns_debug_inject": (C.c_int, [C.c_void_p, C.c_longlong]),
    "dns_debug_stall": (C.c_int, [C.c_void_p]),
    "dns_save": (C.c_int, [C.c_void_p, C.c_char_p]),
    "dns_load": (C.c_int, [C.c_void_p, C.c_char_p]),
    "dns_crc32": (C.c_uint, [C.c_void_p, C.c_size_t, C.c_uint]),
    "dns_debug_f32_from_f64": (C.c_int, [C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p]),
    "dns_measure_fp64_rate": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
})
TRACE_COLS = 8
MLP_PARAMS = 5313
CONTROLLERS = {"I": 0, "PI": 1, "MLP": 2}


def load(path: Optional[str] = None):
    """Load libdns.so (fails loudly if it has not been built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libdns.so not found at {p}; build it with "
                          "`python -m paper_1810_10197_gb300.build`")
    lib = C.CDLL(p)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def declared_symbols():
    """Function names declared in include/dns.h."""
    import re
    txt = open(HEADER_PATH).read()
    return sorted(set(re.findall(r"\b(dns_[a-z0-9_]+)\s*\(", txt)))


# ---- thin module-level wrappers with the C names ----------------------------------------

def _spectral_dev(t, ncomp, shape, what):
    """Address of a device spectral field: a contiguous complex128 CUDA tensor of
    ncomp * nx * ny * (nz/2+1) elements.  Anything else raises ValueError before the library
    is called, so that no kernel reads or writes past a caller's buffer."""
    nx, ny, nz = shape
    want = ncomp * nx * ny * (nz // 2 + 1)
    if not hasattr(t, "data_ptr") or not getattr(t, "is_cuda", False):
        raise ValueError(f"{what}: a CUDA tensor is required")
    if str(t.dtype) != "torch.complex128":
        raise ValueError(f"{what}: dtype complex128 required, got {t.dtype}")
    if t.numel() != want:
        raise ValueError(f"{what}: {t.numel()} elements, expected {want} = {ncomp} x {nx} x {ny} x {nz // 2 + 1}")
    return _ptr(t)


def _ptr(x):
    """Address of a torch tensor or numpy array (contiguous), or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _where(x):
    """0 for device memory (a CUDA tensor), 1 for host memory."""
    if hasattr(x, "is_cuda"):
        return 0 if x.is_cuda else 1
    return 1


def _config(nx, ny=None, nz=None, nu=0.0, precision="fp64", lengths=None):
    cfg = dns_config()
    cfg.nx, cfg.ny, cfg.nz = nx, (nx if ny is None else ny), (nx if nz is None else nz)
    if lengths is not None:
        cfg.lx, cfg.ly, cfg.lz = (float(v) for v in lengths)
    cfg.nu = float(nu)
    cfg.precision = PRECISIONS[precision] \
        if isinstance(precision, str) else int(precision)
    return cfg


class Dns:
    """One libdns context (an nx x ny x nz grid on the current CUDA device)."""

    def __init__(self, nx, ny=None, nz=None, nu=0.0, precision="fp64", forcing=None,
                 lengths=None, stream=None, boussinesq=None, dealias="2/3"):
        """precision: "fp64", "fp32_mixed" (FP32 transforms; k, stage sums and error norm in
        FP64), "fp32" (also k, the stage inputs and the increments in FP32) or "fp32x2"
        (double-word transforms); the state is FP64 in every form (see dns.h dns_precision).
        forcing: (kf, power) constant-power term, or ("rescale", kf) for the post-step band
        rescale.  boussinesq=(kappa, ri) selects the Boussinesq form (state of 4 components);
        dealias="3/2" selects the padding rule (state of nx x ny x nz frequencies)."""
        lib = load()
        ny = nx if ny is None else ny
        nz = nx if nz is None else nz
        cfg = dns_config()
        cfg.nx, cfg.ny, cfg.nz = nx, ny, nz
        if lengths is not None:
            cfg.lx, cfg.ly, cfg.lz = (float(v) for v in lengths)
        cfg.nu = float(nu)
        cfg.precision = PRECISIONS[precision] \
            if isinstance(precision, str) else int(precision)
        if forcing is not None:
            # (kf, power): constant-power right-hand-side term; ("rescale", kf): the
            # post-step band rescale of Section 3.3.1
            if isinstance(forcing[0], str):
                if forcing[0] != "rescale":
                    raise ValueError(f"unknown forcing {forcing[0]!r}")
                cfg.forcing.kind = 2
                cfg.forcing.kf, cfg.forcing.power = float(forcing[1]), 0.0
            else:
                cfg.forcing.kind = 1
                cfg.forcing.kf, cfg.forcing.power = float(forcing[0]), float(forcing[1])
        cfg.dealias = {"2/3": 0, "3/2": 1}[dealias]
        h = C.c_void_p()
        if boussinesq is not None:
            st = lib.dns_create_boussinesq(C.byref(cfg), float(boussinesq[0]), float(boussinesq[1]),
                                           C.byref(h))
        else:
            st = lib.dns_create_ex(C.byref(cfg), C.byref(h))
        if st != DNS_OK:
            raise DnsError(st, "dns_create")
        self.ncomp = 4 if boussinesq is not None else 3
        self._lib = lib
        self._h = h
        self.shape = (nx, ny, nz)
        self.nzh = nz // 2 + 1
        if stream is not None:
            self.set_stream(stream)

    # lifetime
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.dns_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != DNS_OK:
            msg = self._lib.dns_last_error(self._h)
            raise DnsError(st, f"{what}: {msg.decode() if msg else ''}")

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an int handle, or None (legacy default stream)."""
        h = getattr(stream, "cuda_stream", stream)
        self._check(self._lib.dns_set_stream(self._h, C.c_void_p(h) if h else None), "dns_set_stream")

    def set_state(self, uhat, t=0.0):
        self._check(self._lib.dns_set_state(self._h, C.c_void_p(_ptr(uhat)), _where(uhat), float(t)),
                    "dns_set_state")

    def get_state(self, out=None):
        """Current state; into `out` (device tensor or host array) or a new numpy array."""
        if out is None:
            out = np.empty((self.ncomp,) + self.shape[:2] + (self.nzh,), dtype=np.complex128)
        self._check(self._lib.dns_get_state(self._h, C.c_void_p(_ptr(out)), _where(out)), "dns_get_state")
        return out

    def rhs(self, uhat_dev, f_dev):
        a = _spectral_dev(uhat_dev, self.ncomp, self.shape, "dns_rhs input")
        b = _spectral_dev(f_dev, self.ncomp, self.shape, "dns_rhs output")
        self._check(self._lib.dns_rhs(self._h, C.c_void_p(a), C.c_void_p(b)), "dns_rhs")

    def step(self, method, h, rtol=1e-6, atol=1e-6, t_end=float("inf")):
        info = dns_step_info()
        m = METHODS[method] if isinstance(method, str) else int(method)
        self._check(self._lib.dns_step(self._h, m, float(h), float(rtol), float(atol), float(t_end),
                                       C.byref(info)), "dns_step")
        return info

    def integrate(self, t_end, method, rtol=1e-6, atol=1e-6, h0=0.0, max_rejects=0, check=True):
        info = dns_step_info()
        m = METHODS[method] if isinstance(method, str) else int(method)
        st = self._lib.dns_integrate(self._h, float(t_end), m, float(rtol), float(atol), float(h0),
                                     int(max_rejects), C.byref(info))
        if check:
            self._check(st, "dns_integrate")
        return info if check else (st, info)

    def enqueue_attempts(self, n, method, rtol=1e-6, atol=1e-6, t_end=float("inf"), h0=0.0):
        m = METHODS[method] if isinstance(method, str) else int(method)
        self._check(self._lib.dns_enqueue_attempts(self._h, int(n), m, float(rtol), float(atol),
                                                   float(t_end), float(h0)), "dns_enqueue_attempts")

    def info(self):
        info = dns_step_info()
        self._check(self._lib.dns_get_info(self._h, C.byref(info)), "dns_get_info")
        return info

    def diagnostics(self):
        E, O, eps = C.c_double(), C.c_double(), C.c_double()
        self._check(self._lib.dns_diagnostics(self._h, C.byref(E), C.byref(O), C.byref(eps)),
                    "dns_diagnostics")
        return E.value, O.value, eps.value

    def profile_enable(self, on=True):
        self._check(self._lib.dns_profile_enable(self._h, 1 if on else 0), "dns_profile_enable")

    def profile(self):
        out = {}
        for i in range(self._lib.dns_profile_count(self._h)):
            name, n, ms = C.c_char_p(), C.c_longlong(), C.c_double()
            self._check(self._lib.dns_profile_get(self._h, i, C.byref(name), C.byref(n), C.byref(ms)),
                        "dns_profile_get")
            if n.value:
                out[name.value.decode()] = (n.value, ms.value)
        return out

    def spectrum(self):
        """Shell energy spectrum E(k), k = 0..kmax, of the current state."""
        n = C.c_int()
        self._check(self._lib.dns_spectrum(self._h, None, 0, C.byref(n)), "dns_spectrum")
        out = np.empty(n.value)
        self._check(self._lib.dns_spectrum(self._h, C.c_void_p(out.ctypes.data), n.value, C.byref(n)),
                    "dns_spectrum")
        return out

    def autotune(self, reps=3):
        v = (C.c_int * 2)()
        self._check(self._lib.dns_autotune(self._h, int(reps), v), "dns_autotune")
        return tuple(v)

    def set_tiles(self, var_py, var_p3):
        self._check(self._lib.dns_set_tiles(self._h, int(var_py), int(var_p3)), "dns_set_tiles")

    def set_trace(self, capacity, diagnostics=False):
        self._check(self._lib.dns_set_trace(self._h, int(capacity), 1 if diagnostics else 0), "dns_set_trace")

    def trace(self):
        """Attempt records as an (n, 8) array: t, h, err, accepted, n_rhs, E, Omega, eps."""
        n = C.c_longlong()
        self._check(self._lib.dns_trace(self._h, None, 0, C.byref(n)), "dns_trace")
        out = np.empty((n.value, TRACE_COLS))
        if n.value:
            self._check(self._lib.dns_trace(self._h, C.c_void_p(out.ctypes.data), n.value, C.byref(n)),
                        "dns_trace")
        return out

    def set_controller(self, kind, params_dev=None):
        k = CONTROLLERS[kind] if isinstance(kind, str) else int(kind)
        self._check(self._lib.dns_set_controller(self._h, k, C.c_void_p(_ptr(params_dev)) if params_dev is not None
                                                 else None), "dns_set_controller")

    def debug_inject(self, rhs_index):
        self._check(self._lib.dns_debug_inject(self._h, int(rhs_index)), "dns_debug_inject")

    def debug_stall(self):
        self._check(self._lib.dns_debug_stall(self._h), "dns_debug_stall")

    def debug_poison(self, on=True):
        self._check(self._lib.dns_debug_poison(self._h, 1 if on else 0), "dns_debug_poison")

    def save(self, path):
        self._check(self._lib.dns_save(self._h, os.fsencode(path)), "dns_save")

    def load(self, path):
        self._check(self._lib.dns_load(self._h, os.fsencode(path)), "dns_load")

    def query(self):
        K = (C.c_int * 3)()
        nb = C.c_size_t()
        self._check(self._lib.dns_query(self._h, K, C.byref(nb)), "dns_query")
        return tuple(K), nb.value


def dns_crc32(data: bytes, crc: int = 0) -> int:
    """CRC-32 of the checkpoint trailer (host code, no GPU needed)."""
    buf = C.create_string_buffer(bytes(data), len(data))
    return int(load().dns_crc32(buf, len(data), crc))


def dns_measure_fp64_rate(stream=None):
    """(DFMA, DADD) thread instructions per second of the current device's FP64 pipe."""
    a, b = C.c_double(), C.c_double()
    h = getattr(stream, "cuda_stream", stream)
    st = load().dns_measure_fp64_rate(C.c_void_p(h) if h else None, C.byref(a), C.byref(b))
    if st != DNS_OK:
        raise DnsError(st, "dns_measure_fp64_rate")
    return a.value, b.value


def dns_debug_f32_from_f64(x_dev, y_dev, stream=None):
    """The integer-bit FP64-to-FP32 conversion of the single-precision kernels (test hook)."""
    h = getattr(stream, "cuda_stream", stream)
    st = load().dns_debug_f32_from_f64(C.c_void_p(_ptr(x_dev)), C.c_void_p(_ptr(y_dev)), int(x_dev.numel()),
                                       C.c_void_p(h) if h else None)
    if st != 0:
        raise DnsError(st, "dns_debug_f32_from_f64")


def dns_rhs_noalloc(nx, ny, nz, nu, uhat_dev, f_dev, stream=None):
    """dns_rhs without a context or device allocation (grids up to 32^3); returns the status."""
    lib = load()
    h = getattr(stream, "cuda_stream", stream)
    shape = (int(nx), int(ny), int(nz))
    a = _spectral_dev(uhat_dev, 3, shape, "dns_rhs_noalloc input")
    b = _spectral_dev(f_dev, 3, shape, "dns_rhs_noalloc output")
    return lib.dns_rhs_noalloc(shape[0], shape[1], shape[2], float(nu), C.c_void_p(a),
                               C.c_void_p(b), C.c_void_p(h) if h else None)


def _st(stream):
    h = getattr(stream, "cuda_stream", stream)
    return C.c_void_p(h) if h else None


def dns_mlp_forward(params, x, y, stream=None):
    """y[b] = network(x[b]) for device float32 tensors params[5313], x[n,16], y[n]."""
    return load().dns_mlp_forward(C.c_void_p(_ptr(params)), C.c_void_p(_ptr(x)), int(x.shape[0]),
                                  C.c_void_p(_ptr(y)), _st(stream))


def dns_mlp_loss_grad(params, x, t, grad, loss, stream=None):
    return load().dns_mlp_loss_grad(C.c_void_p(_ptr(params)), C.c_void_p(_ptr(x)), C.c_void_p(_ptr(t)),
                                    int(x.shape[0]), C.c_void_p(_ptr(grad)), C.c_void_p(_ptr(loss)),
                                    _st(stream))


def dns_mlp_train(params, x, t, steps, batch=128, lr=1e-3, seed=0, loss_hist=None, stream=None):
    return load().dns_mlp_train(C.c_void_p(_ptr(params)), C.c_void_p(_ptr(x)), C.c_void_p(_ptr(t)),
                                int(x.shape[0]), int(steps), int(batch), float(lr), int(seed) & 0xFFFFFFFF,
                                C.c_void_p(_ptr(loss_hist)) if loss_hist is not None else None, _st(stream))


class _Borrowed(Dns):
    """A context owned by a batch (not destroyed by Python)."""

    def __init__(self, lib, handle, shape):
        self._lib = lib
        self._h = handle
        self.shape = tuple(shape)
        self.nzh = shape[2] // 2 + 1
        self.ncomp = 3

    def close(self):
        self._h = C.c_void_p()


class DnsBatch:
    """An ensemble of independent simulations advanced by one graph launch."""

    def __init__(self, configs):
        """configs: list of dicts with keys nx[, ny, nz, nu, precision, lengths]."""
        lib = load()
        arr = (dns_config * len(configs))()
        for i, c in enumerate(configs):
            arr[i] = _config(**c)
        h = C.c_void_p()
        st = lib.dns_create_batch(len(configs), arr, C.byref(h))
        if st != DNS_OK:
            raise DnsError(st, "dns_create_batch")
        self._lib, self._h, self.n = lib, h, len(configs)
        self.instances = []
        for i, c in enumerate(configs):
            ch = C.c_void_p()
            lib.dns_batch_context(h, i, C.byref(ch))
            nx = c["nx"]
            self.instances.append(_Borrowed(lib, ch, (nx, c.get("ny") or nx, c.get("nz") or nx)))

    def integrate(self, method, t_end, rtol, atol, h0, check=True):
        n = self.n
        D = C.c_double * n
        info = (dns_step_info * n)()
        m = METHODS[method] if isinstance(method, str) else int(method)
        st = self._lib.dns_integrate_batch(self._h, m, D(*t_end), D(*rtol), D(*atol), D(*h0), info)
        if check and st != DNS_OK:
            raise DnsError(st, "dns_integrate_batch: " + (self._lib.dns_batch_last_error(self._h) or b"").decode())
        return list(info) if check else (st, list(info))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            for inst in self.instances:
                inst.close()
            self._lib.dns_destroy_batch(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
