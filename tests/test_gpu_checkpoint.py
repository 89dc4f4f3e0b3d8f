"""Checkpoint and resume (dns_save / dns_load) and the band rescale forcing of Section 3.3.1.

A resumed run must reproduce the uninterrupted one bit for bit: the checkpoint carries the
state, the carried-over k_1 of a first-same-as-last pair and the controller's state.  The
rescale forcing is compared with the oracle's integrate(..., post_step=rescale_band) at the
FP64 bound of the other integration tests (1e-12 relative L2, decisions identical).
"""
import os
import struct
import zlib

import numpy as np
import pytest

import synthetic as syn
from oracle import diag, rk
from oracle import spectral as sp
from tests.gpu_helpers import lib_ready, rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu

HEADER_BYTES = 372      # fixed part of the version-1 layout declared in dns.h


@pytest.fixture(scope="module", autouse=True)
def _lib():
    require_gpu()
    lib_ready()


def make(shape, uh, nu, forcing=None, t0=0.0, precision="fp64"):
    from paper_1810_10197_gb300 import Dns
    d = Dns(*shape, nu=nu, forcing=forcing, precision=precision)
    d.set_state(to_dev(uh), t0)
    return d


def _hit(shape, seed=3):
    g = sp.Grid(*shape)
    return g, g.dealias(syn.random_solenoidal_hat(*shape, seed=seed, k0=3.0))


def _same(a, b):
    return a.tobytes() == b.tobytes()


@pytest.mark.parametrize("method,ctrl,h0,prec", [("BS5_ADAPTIVE", "I", 0.5, "fp64"), ("DP5_ADAPTIVE", "PI", 0.5, "fp64"),
                                                 ("BS5_FIXED", "I", 2e-3, "fp64"), ("RK4", "I", 2e-3, "fp64"),
                                                 ("BS5_ADAPTIVE", "I", 0.5, "fp32_mixed"),
                                                 ("BS5_ADAPTIVE", "PI", 0.5, "fp32")])
def test_resume_is_bit_for_bit(tmp_path, method, ctrl, h0, prec):
    # 10 attempts in one context == 5 attempts, save, load into a fresh context, 5 attempts.
    # The large h0 of the adaptive runs forces rejections inside the first five attempts.
    # fp32: the carried k_1 is held in FP32 on the device and written widened (exactly) to the
    # file, so the resumed run is bit-identical as well.
    shape, nu, tol = (32, 32, 32), 0.01, 1e-7
    g, uh = _hit(shape)
    a = make(shape, uh, nu, precision=prec)
    a.set_controller(ctrl)
    a.enqueue_attempts(10, method, tol, tol, h0=h0)
    ia, ua = a.info(), a.get_state()
    b = make(shape, uh, nu, precision=prec)
    b.set_controller(ctrl)
    b.enqueue_attempts(5, method, tol, tol, h0=h0)
    mid = b.info()
    path = str(tmp_path / "mid.ckpt")
    b.save(path)
    c = make(shape, np.zeros_like(uh), nu, precision=prec)     # a different state, overwritten by the load
    c.load(path)
    ic0 = c.info()
    assert (ic0.t, ic0.h_next, ic0.n_rhs, ic0.n_acc, ic0.n_rej) == \
        (mid.t, mid.h_next, mid.n_rhs, mid.n_acc, mid.n_rej)
    assert _same(c.get_state(), b.get_state())
    c.enqueue_attempts(5, method, tol, tol, h0=0.0)
    ic, uc = c.info(), c.get_state()
    if method.endswith("ADAPTIVE"):
        assert mid.n_rej >= 1
    assert _same(uc, ua)
    assert (ic.t, ic.h_next, ic.err, ic.n_rhs, ic.n_acc, ic.n_rej) == \
        (ia.t, ia.h_next, ia.err, ia.n_rhs, ia.n_acc, ia.n_rej)


def test_checkpoint_file_layout(tmp_path):
    shape, nu = (16, 16, 32), 0.02
    g, uh = _hit(shape, seed=5)
    d = make(shape, uh, nu)
    d.enqueue_attempts(3, "BS5_ADAPTIVE", 1e-6, 1e-6, h0=0.01)
    info = d.info()
    path = str(tmp_path / "c.ckpt")
    d.save(path)
    raw = open(path, "rb").read()
    assert raw[:8] == b"DNSCKPT1"
    assert struct.unpack_from("<I6i", raw, 8) == (1, 16, 16, 32, 0, 3, 0)
    (crc,) = struct.unpack_from("<I", raw, len(raw) - 4)
    assert crc == zlib.crc32(raw[:-4])
    # controller block: t is the first double after the forcing fields
    off_ctrl = 8 + 4 + 24 + 48 + 4 + 16
    assert struct.unpack_from("<d", raw, off_ctrl)[0] == info.t
    K = [(n - 1) // 3 for n in shape]
    M = (2 * K[0] + 1) * (2 * K[1] + 1) * (K[2] + 1)
    assert struct.unpack_from("<q", raw, HEADER_BYTES - 8)[0] == M
    k1_valid = struct.unpack_from("<i", raw, off_ctrl + 11 * 8 + 4)[0]
    assert k1_valid == 1            # BS5 after an attempt carries k_1 over
    assert len(raw) == HEADER_BYTES + 2 * 3 * M * 16 + 4
    # the state section is the retained box of the current state, kz fastest
    state = np.frombuffer(raw, dtype=np.complex128, count=3 * M, offset=HEADER_BYTES)
    full = d.get_state()
    ix = np.r_[0:K[0] + 1, shape[0] - K[0]:shape[0]]
    iy = np.r_[0:K[1] + 1, shape[1] - K[1]:shape[1]]
    box = full[:, ix][:, :, iy][:, :, :, :K[2] + 1]
    assert _same(state, np.ascontiguousarray(box).ravel())


def test_load_rejects_bad_files_and_keeps_the_context(tmp_path):
    from paper_1810_10197_gb300 import DnsError
    shape, nu = (16, 16, 16), 0.02
    g, uh = _hit(shape, seed=8)
    d = make(shape, uh, nu)
    d.enqueue_attempts(2, "BS5_ADAPTIVE", 1e-6, 1e-6, h0=0.01)
    good = str(tmp_path / "good.ckpt")
    d.save(good)
    raw = bytearray(open(good, "rb").read())
    e = make(shape, 0.5 * uh, nu, t0=3.0)
    before, info0 = e.get_state(), e.info()
    cases = {}
    flipped = bytearray(raw)
    flipped[HEADER_BYTES + 100] ^= 0x01
    cases["crc"] = bytes(flipped)
    cases["truncated"] = bytes(raw[:-20])
    cases["magic"] = b"NOTACKPT" + bytes(raw[8:])
    for name, blob in cases.items():
        p = str(tmp_path / f"{name}.ckpt")
        open(p, "wb").write(blob)
        with pytest.raises(DnsError) as ex:
            e.load(p)
        assert ex.value.status == 1, name          # DNS_ERR_ARG
    with pytest.raises(DnsError) as ex:
        e.load(str(tmp_path / "missing.ckpt"))
    assert ex.value.status == 1
    # another grid
    g2, uh2 = _hit((16, 16, 32))
    f = make((16, 16, 32), uh2, nu)
    with pytest.raises(DnsError) as ex:
        f.load(good)
    assert ex.value.status == 1
    assert _same(e.get_state(), before) and e.info().t == info0.t
    # and the good file still loads
    e.load(good)
    assert _same(e.get_state(), d.get_state())


@pytest.mark.parametrize("method,h0", [("BS5_ADAPTIVE", 0.01), ("RK4", 0.01)])
def test_band_rescale_forcing_matches_oracle(method, h0):
    shape, nu, kf, T, tol = (32, 32, 32), 0.02, 2.5, 0.15, 1e-7
    g, uh = _hit(shape, seed=11)
    e0 = diag.energy(g, uh)
    ref = rk.integrate(lambda y: sp.rhs(g, y, nu), uh, 0.0, T, method, h0, tol, tol,
                       nmodes=g.nmodes_half, post_step=lambda a, b: sp.rescale_band(g, a, b, kf))
    d = make(shape, uh, nu, forcing=("rescale", kf))
    info = d.integrate(T, method, tol, tol, h0=h0)
    assert info.t == T
    assert (info.n_acc, info.n_rej, info.n_rhs) == (ref.n_acc, ref.n_rej, ref.n_rhs)
    u = d.get_state()
    assert rel_l2(u, ref.u) < 1e-12
    assert abs(diag.energy(g, u) - e0) < 1e-12 * e0


def test_forced_spinup_resumed_as_decaying_run(tmp_path):
    # Section 3.3.2 protocol: spin up with the band rescale, then restart without forcing
    shape, nu, kf, t_mid, t_end, tol = (32, 32, 32), 0.02, 2.5, 0.1, 0.2, 1e-7
    g, uh = _hit(shape, seed=13)
    r1 = rk.integrate(lambda y: sp.rhs(g, y, nu), uh, 0.0, t_mid, "BS5_ADAPTIVE", 0.01, tol, tol,
                      nmodes=g.nmodes_half, post_step=lambda a, b: sp.rescale_band(g, a, b, kf))
    r2 = rk.integrate(lambda y: sp.rhs(g, y, nu), r1.u, r1.t, t_end, "BS5_ADAPTIVE", r1.h_next, tol, tol,
                      nmodes=g.nmodes_half)
    a = make(shape, uh, nu, forcing=("rescale", kf))
    a.integrate(t_mid, "BS5_ADAPTIVE", tol, tol, h0=0.01)
    path = str(tmp_path / "spun_up.ckpt")
    a.save(path)
    b = make(shape, np.zeros_like(uh), nu)
    b.load(path)
    info = b.integrate(t_end, "BS5_ADAPTIVE", tol, tol, h0=0.0)
    assert info.t == t_end
    assert (info.n_acc, info.n_rej) == (r1.n_acc + r2.n_acc, r1.n_rej + r2.n_rej)
    assert rel_l2(b.get_state(), r2.u) < 1e-12
    assert os.path.getsize(path) > HEADER_BYTES
