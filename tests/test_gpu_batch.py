"""Batched ensembles: uneven-size independent simulations advanced by one graph launch
(dns_integrate_batch) must reproduce, instance by instance, what the oracle (and a single
context) compute: identical accept/reject counts and 1e-12 relative L2 state (FP64)."""
import numpy as np
import pytest

import synthetic as syn
from oracle import rk
from oracle import spectral as sp
from tests.gpu_helpers import rel_max, lib_ready, rel_l2, require_gpu, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    require_gpu()
    lib_ready()


def test_uneven_batch_matches_oracle_per_instance():
    from paper_1810_10197_gb300.dns import DnsBatch
    specs = [(16, 0.02, 3.0, 0.20), (24, 0.005, 2.0, 0.30), (32, 0.01, 5.0, 0.25), (16, 0.003, 4.0, 0.15),
             (32, 0.002, 2.5, 0.10)]
    cfgs = [dict(nx=n, nu=nu) for (n, nu, _, _) in specs]
    b = DnsBatch(cfgs)
    fields = []
    for i, (n, nu, k0, _) in enumerate(specs):
        g = sp.Grid(n, n, n)
        uh = g.dealias(syn.random_solenoidal_hat(n, n, n, seed=100 + i, k0=k0))
        fields.append(uh)
        b.instances[i].set_state(to_dev(uh), 0.0)
    tols = [1e-7, 1e-6, 1e-8, 1e-7, 1e-6]
    t_end = [s[3] for s in specs]
    infos = b.integrate("BS5_ADAPTIVE", t_end, tols, tols, [0.01] * len(specs))
    for i, (n, nu, _, T) in enumerate(specs):
        g = sp.Grid(n, n, n)
        ref = rk.integrate(lambda y, g=g, nu=nu: sp.rhs(g, y, nu), fields[i], 0.0, T, "BS5_ADAPTIVE",
                           0.01, tols[i], tols[i], nmodes=g.nmodes_half)
        assert infos[i].t == T
        assert (infos[i].n_acc, infos[i].n_rej, infos[i].n_rhs) == (ref.n_acc, ref.n_rej, ref.n_rhs)
        assert rel_l2(b.instances[i].get_state(), ref.u) < 1e-12
    # a second launch of the cached graph continues every instance to a later time
    t2 = [t + 0.05 for t in t_end]
    infos2 = b.integrate("BS5_ADAPTIVE", t2, tols, tols, [0.0] * len(specs))
    assert all(inf.t == t for inf, t in zip(infos2, t2))
    assert all(i2.n_acc > i1.n_acc for i1, i2 in zip(infos, infos2))
    b.close()


def test_batch_with_finished_instances_is_a_noop():
    from paper_1810_10197_gb300.dns import DnsBatch
    b = DnsBatch([dict(nx=16, nu=0.01), dict(nx=16, nu=0.01)])
    for i in range(2):
        b.instances[i].set_state(to_dev(syn.taylor_green_3d_hat(16, 16, 16)), 1.0)
    infos = b.integrate("BS5_ADAPTIVE", [1.0, 0.5], [1e-6, 1e-6], [1e-6, 1e-6], [0.01, 0.01])
    assert all(inf.n_rhs == 0 and inf.t == 1.0 for inf in infos)
    b.close()


@pytest.mark.parametrize("shape,precision", [((32, 32, 32), "fp64"), ((64, 48, 64), "fp32_mixed"),
                                             ((96, 96, 96), "fp64")])
def test_tile_variants_give_identical_results_and_autotune_picks_one(shape, precision):
    import torch
    from paper_1810_10197_gb300 import Dns
    uh = syn.random_solenoidal_hat(*shape, seed=7, k0=3.0)
    d = Dns(*shape, nu=0.01, precision=precision)
    u = to_dev(uh)
    outs = []
    for v in ((0, 0), (1, 0), (0, 1), (1, 1), (0, 2), (1, 3)):
        d.set_tiles(*v)
        f = torch.empty_like(u)
        d.rhs(u, f)
        torch.cuda.synchronize()
        outs.append(f.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])      # the same arithmetic per line, any tiling
    # z pass codes 4 and 5: the register-resident FP32 kernel (single-precision forms, nz = 64,
    # 128, 256; elsewhere codes 0 and 1) with paired or scalar FP32 instructions (the scalar
    # form lets the compiler fuse some products into FMAs): against each other and against
    # codes 0..3 (another schedule) they agree to FP32 rounding
    rr = []
    for v in ((0, 4), (1, 5)):
        d.set_tiles(*v)
        f = torch.empty_like(u)
        d.rhs(u, f)
        torch.cuda.synchronize()
        rr.append(f.cpu().numpy())
    if precision == "fp64":
        assert np.array_equal(rr[0], outs[0]) and np.array_equal(rr[1], outs[0])
    else:
        assert rel_max(rr[1], rr[0]) < 2e-5 and rel_max(rr[0], outs[0]) < 2e-5
    vpy, vp3 = d.autotune(reps=2)
    assert vpy in (0, 1) and vp3 in range(6)   # z pass: bit 0 tile, bit 1 element copies, bit 2 RR kernel
    d.close()


def test_mixed_precision_batch_matches_single_contexts_bitwise():
    # instances of different forms (FP64, FP32-mixed, fp32 with its FP32 k and stage-input
    # slots) in one graph launch: each runs the same kernels in the same order as a single
    # context of its form, so the states agree bit for bit
    from paper_1810_10197_gb300 import Dns
    from paper_1810_10197_gb300.dns import DnsBatch
    specs = [(32, "fp32", 0.01, 0.2), (24, "fp32_mixed", 0.005, 0.15), (16, "fp64", 0.02, 0.25)]
    b = DnsBatch([dict(nx=n, nu=nu, precision=p) for (n, p, nu, _) in specs])
    fields = []
    for i, (n, p, nu, _) in enumerate(specs):
        g = sp.Grid(n, n, n)
        uh = g.dealias(syn.random_solenoidal_hat(n, n, n, seed=200 + i, k0=3.0))
        fields.append(uh)
        b.instances[i].set_state(to_dev(uh), 0.0)
    tols = [1e-6, 1e-6, 1e-7]
    infos = b.integrate("BS5_ADAPTIVE", [s[3] for s in specs], tols, tols, [0.01] * 3)
    for i, (n, p, nu, T) in enumerate(specs):
        d = Dns(n, nu=nu, precision=p)
        d.set_state(to_dev(fields[i]), 0.0)
        info = d.integrate(T, "BS5_ADAPTIVE", tols[i], tols[i], h0=0.01)
        assert (infos[i].t, infos[i].n_acc, infos[i].n_rej, infos[i].n_rhs) == (info.t, info.n_acc, info.n_rej, info.n_rhs)
        assert b.instances[i].get_state().tobytes() == d.get_state().tobytes()
        d.close()
    b.close()
