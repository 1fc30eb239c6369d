"""Batched scaling (sa_batch_scale, one persistent launch over many small instances)
against the FP64 oracle, and each instance alone equal to the same instance inside the
batch (the result of one instance does not depend on its neighbours)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1104_3830_gb300 import _lib as L
from paper_1104_3830_gb300 import api
from paper_1104_3830_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_3830_gb300 import build
    build.build()
    c = api.sa_create(0)
    yield c
    c.close()


def batch_scale(ctx, mats, ps, tol=1e-6, sweeps=20000, plan=None):
    """Pack instances as device tensors and run sa_batch_scale; returns (u_list, v_list, sweeps, status)."""
    devs = [api.to_device(m) for m in mats]
    k = len(mats)
    ptrs = torch.tensor([d.data_ptr() for d in devs], dtype=torch.int64, device="cuda")
    ns = torch.tensor([m.shape[0] for m in mats], dtype=torch.int32, device="cuda")
    lds = torch.tensor([d.stride(0) for d in devs], dtype=torch.int64, device="cuda")
    offs_h = np.concatenate([[0], np.cumsum([m.shape[0] for m in mats])[:-1]]).astype(np.int64)
    offs = torch.from_numpy(offs_h).cuda()
    tot = int(sum(m.shape[0] for m in mats))
    u = torch.zeros(tot, dtype=torch.float64, device="cuda")
    v = torch.zeros(tot, dtype=torch.float64, device="cuda")
    sw = np.zeros(k, dtype=np.int32)
    st = np.zeros(k, dtype=np.int32)
    o = L.make_opts(ps, tol, sweeps)
    wt = L.SA_I16 if mats[0].dtype == np.int16 else L.SA_I32
    if plan is not None:
        api.sa_set_batch_plan(ctx, plan)
    try:
        rc = L.lib().sa_batch_scale(ctx.handle, k, ctypes.c_void_p(ptrs.data_ptr()), ctypes.c_void_p(ns.data_ptr()),
                                    ctypes.c_void_p(lds.data_ptr()), ctypes.c_void_p(offs.data_ptr()), wt,
                                    ctypes.byref(o), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                    sw.ctypes.data_as(L._I32P), st.ctypes.data_as(L._I32P))
    finally:
        if plan is not None:
            api.sa_set_batch_plan(ctx, None)
    uh, vh = u.cpu().numpy(), v.cpu().numpy()
    us = [uh[o_:o_ + m.shape[0]] for o_, m in zip(offs_h, mats)]
    vs = [vh[o_:o_ + m.shape[0]] for o_, m in zip(offs_h, mats)]
    return rc, us, vs, sw, st


@pytest.mark.parametrize("dtype", [np.int16, np.int32])
def test_batch_matches_oracle(ctx, dtype):
    sizes = [1, 2, 7, 16, 33, 100, 129, 250, 300, 512, 64, 17]
    mats = [W.uniform(n, 1, 1000, 1000 + k, dtype=dtype) for k, n in enumerate(sizes)]
    ps = [2.0 ** k for k in range(6)]
    rc, us, vs, sw, st = batch_scale(ctx, mats, ps)
    assert rc == 0 and np.all(st == 0), (rc, st)
    for m, u, v in zip(mats, us, vs):
        b = oracle.log_weights(m.astype(np.int64))
        r, c = oracle.sums(b, ps[-1], u, v)
        err = max(np.abs(r - 1).max(), np.abs(c - 1).max())
        assert err < 2 * ps[-1] * np.log(2) * 1e-6 + 4e-6, (m.shape, err)
        uo, vo, _, _, sto = oracle.sinkhorn(b, ps, 1e-6, 20000)
        assert sto == 0
        xo = oracle.xmatrix(b, ps[-1], uo, vo)
        xg = oracle.xmatrix(b, ps[-1], u, v)
        assert np.max(np.abs(xg - xo)) < 1e-4


GROUP_PLAN = [(32, "group", 1, 4), (64, "group", 2, 4), (128, "group", 4, 1), (512, "block", 0, 0)]


@pytest.mark.parametrize("dtype", [np.int16, np.int32])
def test_group_path_error_does_not_grow_with_p(ctx, dtype):
    """Instances of n <= 128 run on the group path on the per-step matrix K (float-pair
    exponent once per p step): up to p = 128 their FP64-recomputed sums stay within the bound
    of the per-step path (2e-6), independent of p, unlike the block path's FP32 logarithm
    (about 1.3e-7 p).  Ragged sizes: one row, odd n, every template (n <= 32, 64, 128) and
    both sides of each boundary."""
    sizes = [1, 3, 5, 16, 31, 32, 33, 47, 63, 64, 65, 99, 127, 128]
    mats = [W.uniform(n, 1, 1000, 1100 + n, dtype=dtype) for n in sizes]
    ps = [2.0 ** k for k in range(8)]
    rc, us, vs, sw, st = batch_scale(ctx, mats, ps, sweeps=20000, plan=GROUP_PLAN)
    assert rc in (0, L.SA_E_NOT_CONVERGED), rc
    for m, u, v, s_, c_ in zip(mats, us, vs, sw, st):
        b = oracle.log_weights(m.astype(np.int64))
        uo, vo, swo, rso, sto = oracle.sinkhorn(b, ps, 1e-6, 20000)
        # the same stopping decisions as the oracle's (the cap where it caps)
        assert c_ == (1 if sto == oracle.NOT_CONVERGED else 0), (m.shape, c_, sto)
        if c_ != 0:
            continue
        r, c = oracle.sums(b, ps[-1], u, v)
        err = max(np.abs(r - 1).max(), np.abs(c - 1).max())
        assert err < 2e-6, (m.shape, err)
        xo = oracle.xmatrix(b, ps[-1], uo, vo)
        xg = oracle.xmatrix(b, ps[-1], u, v)
        assert np.all(np.abs(xg - xo) <= 8e-6 * np.maximum(xo, 1.0 / m.shape[0]) + 1e-9), m.shape


def test_group_and_block_paths_agree(ctx):
    """The same small instances through the group path and through the block path (a plan
    with one block bucket): both within their bounds of the oracle's X(p)."""
    sizes = [2, 9, 24, 40, 64, 90, 128]
    mats = [W.uniform(n, 1, 1000, 1200 + n, dtype=np.int16) for n in sizes]
    ps = [1.0, 2.0, 4.0, 8.0]
    rc_w, uw, vw, sww, stw = batch_scale(ctx, mats, ps, plan=GROUP_PLAN)
    rc_b, ub, vb, swb, stb = batch_scale(ctx, mats, ps, plan=[(512, "block", 0, 0)])
    assert rc_w == 0 and rc_b == 0
    for m, a, b_, c, d in zip(mats, uw, vw, ub, vb):
        b = oracle.log_weights(m.astype(np.int64))
        xw = oracle.xmatrix(b, ps[-1], a, b_)
        xb = oracle.xmatrix(b, ps[-1], c, d)
        assert np.max(np.abs(xw - xb)) < 2 * ps[-1] * np.log(2) * 1e-6 + 1e-5


REGS_PLAN = [(32, "regs", 1, 4), (64, "regs", 4, 2), (128, "regs", 16, 1), (512, "block", 0, 0)]


@pytest.mark.parametrize("dtype", [np.int16, np.int32])
def test_register_path_matches_oracle(ctx, dtype):
    """The register path (K in registers during the sweeps; rows and columns split over 1,
    2 or 4 lanes) on every shape: the oracle's stopping decisions, X(p) within 8e-6 of the
    oracle's entries and FP64 sums within 2e-6 up to p = 128."""
    sizes = [1, 2, 7, 31, 32, 33, 50, 64, 65, 100, 128]
    mats = [W.uniform(n, 1, 1000, 1500 + n, dtype=dtype) for n in sizes]
    ps = [2.0 ** k for k in range(8)]
    rc, us, vs, sw, st = batch_scale(ctx, mats, ps, plan=REGS_PLAN)
    assert rc in (0, L.SA_E_NOT_CONVERGED), rc
    for m, u, v, c_ in zip(mats, us, vs, st):
        b = oracle.log_weights(m.astype(np.int64))
        uo, vo, swo, rso, sto = oracle.sinkhorn(b, ps, 1e-6, 20000)
        assert c_ == (1 if sto == oracle.NOT_CONVERGED else 0), (m.shape, c_, sto)
        if c_ != 0:
            continue
        r, c = oracle.sums(b, ps[-1], u, v)
        assert max(np.abs(r - 1).max(), np.abs(c - 1).max()) < 2e-6, m.shape
        xo = oracle.xmatrix(b, ps[-1], uo, vo)
        xg = oracle.xmatrix(b, ps[-1], u, v)
        assert np.all(np.abs(xg - xo) <= 8e-6 * np.maximum(xo, 1.0 / m.shape[0]) + 1e-9), m.shape


def test_register_path_shapes(ctx):
    """Shapes the register path does not have are refused; the groups per block do not change
    an instance's result (bit-identical), and a zero column is reported as non-finite."""
    for bad in ([(64, "regs", 1, 4), (512, "block", 0, 0)],      # one warp cannot hold n <= 64
                [(128, "regs", 8, 1), (512, "block", 0, 0)],     # eight warps cannot hold n <= 128
                [(32, "regs", 4, 8), (512, "block", 0, 0)]):     # 32 warps per block
        with pytest.raises(api.SaError):
            api.sa_set_batch_plan(ctx, bad)
    mats = [W.uniform(n, 1, 1000, 1600 + n, dtype=np.int16) for n in (5, 20, 32, 40, 64, 90)]
    ps = [1.0, 2.0, 4.0]
    rc0, u0, v0, sw0, _ = batch_scale(ctx, mats, ps, plan=REGS_PLAN)
    rc1, u1, v1, sw1, _ = batch_scale(ctx, mats, ps, plan=[(32, "regs", 1, 1), (64, "regs", 4, 4),
                                                           (128, "regs", 16, 1), (512, "block", 0, 0)])
    assert rc0 == 0 and rc1 == 0 and np.array_equal(sw0, sw1)
    for a, b, c, d in zip(u0, v0, u1, v1):
        assert np.array_equal(a, c) and np.array_equal(b, d)
    z = W.uniform(30, 1, 1000, 1700, dtype=np.int16)
    z[:, 7] = 0
    rc, *_, st = batch_scale(ctx, [z, mats[0]], ps, plan=REGS_PLAN)
    assert rc == L.SA_E_NONFINITE and st[0] == -6 and st[1] == 0


KROWS_PLAN = [(128, "regs", 16, 1), (512, "krows", 0, 0)]


@pytest.mark.parametrize("dtype", [np.int16, np.int32])
def test_krows_path_matches_oracle(ctx, dtype):
    """The K rows path (n up to 512, K in a global slot per block, warps on whole rows) on
    its three widths (n <= 128, 256, 512) and ragged sizes: X(p) within 8e-6 of the oracle's
    entries and FP64 sums within 2e-6 up to p = 64, independent of p."""
    sizes = [129, 130, 200, 255, 256, 257, 300, 511, 512]
    mats = [W.uniform(n, 1, 1000, 1800 + n, dtype=dtype) for n in sizes]
    ps = [2.0 ** k for k in range(7)]
    rc, us, vs, sw, st = batch_scale(ctx, mats, ps, plan=KROWS_PLAN)
    assert rc in (0, L.SA_E_NOT_CONVERGED), rc
    for m, u, v, c_ in zip(mats, us, vs, st):
        b = oracle.log_weights(m.astype(np.int64))
        uo, vo, swo, rso, sto = oracle.sinkhorn(b, ps, 1e-6, 20000)
        assert c_ == (1 if sto == oracle.NOT_CONVERGED else 0), (m.shape, c_, sto)
        if c_ != 0:
            continue
        r, c = oracle.sums(b, ps[-1], u, v)
        assert max(np.abs(r - 1).max(), np.abs(c - 1).max()) < 2e-6, m.shape
        xo = oracle.xmatrix(b, ps[-1], uo, vo)
        xg = oracle.xmatrix(b, ps[-1], u, v)
        assert np.all(np.abs(xg - xo) <= 8e-6 * np.maximum(xo, 1.0 / m.shape[0]) + 1e-9), m.shape
    # alone equals in the batch (one program per instance), and a lost column is reported
    rc1, u1, v1, sw1, st1 = batch_scale(ctx, [mats[4]], ps, plan=KROWS_PLAN)
    assert sw1[0] == sw[4] and np.array_equal(u1[0], us[4]) and np.array_equal(v1[0], vs[4])
    z = mats[0].copy()
    z[:, 5] = 0
    rc2, *_, st2 = batch_scale(ctx, [z, mats[1]], ps, plan=KROWS_PLAN)
    assert rc2 == L.SA_E_NONFINITE and st2[0] == -6 and st2[1] == 0


def test_batch_not_converged_like_oracle(ctx):
    # small uniform instances at p = 128 are nearly decomposable: the oracle hits the
    # cap on exactly these, and so must the batch (status 1, SA_E_NOT_CONVERGED overall)
    sizes = [7, 16, 17, 100, 300]
    mats = [W.uniform(n, 1, 1000, 1000 + k, dtype=np.int16) for k, n in zip([2, 3, 11, 5, 8], sizes)]
    ps = [2.0 ** k for k in range(8)]
    rc, us, vs, sw, st = batch_scale(ctx, mats, ps, sweeps=3000)
    assert rc == L.SA_E_NOT_CONVERGED
    for m, s in zip(mats, st):
        b = oracle.log_weights(m.astype(np.int64))
        sto = oracle.sinkhorn(b, ps, 1e-6, 3000)[4]
        assert s == (1 if sto == oracle.NOT_CONVERGED else 0), (m.shape, s, sto)


def test_alone_equals_in_batch(ctx):
    mats = [W.uniform(n, 1, 1000, 2000 + n, dtype=np.int16) for n in (40, 300, 120, 512, 90)]
    ps = [1.0, 2.0, 4.0, 8.0, 16.0]
    rc, us, vs, sw, st = batch_scale(ctx, mats, ps)
    assert rc == 0
    for k, m in enumerate(mats):
        rc1, u1, v1, sw1, st1 = batch_scale(ctx, [m], ps)
        assert rc1 == 0
        # same instance, same block program: bit-identical potentials and sweep counts
        assert sw1[0] == sw[k]
        assert np.array_equal(u1[0], us[k]) and np.array_equal(v1[0], vs[k])


def test_plans_are_checked_and_applied(ctx):
    """Bad plans are refused; plans of several group buckets with different launch shapes
    give each instance the result of the same warps per instance (the group path's program
    per instance does not depend on the bucket or the groups per block: bit-identical)."""
    for bad in ([(64, "group", 1, 4)],                                     # does not reach 512
                [(256, "group", 4, 1), (512, "block", 0, 0)],              # group path beyond 128
                [(32, "group", 3, 1), (512, "block", 0, 0)],               # 3 warps per instance
                [(32, "group", 4, 4), (512, "block", 0, 0)],               # 16 warps per block
                [(64, "block", 0, 0), (32, "group", 1, 4), (512, "block", 0, 0)]):   # not increasing
        with pytest.raises(api.SaError):
            api.sa_set_batch_plan(ctx, bad)
    sizes = [5, 12, 20, 30, 40, 50, 60, 64, 70, 100, 128, 200]
    mats = [W.uniform(n, 1, 1000, 1300 + n, dtype=np.int16) for n in sizes]
    ps = [1.0, 2.0, 4.0, 8.0]
    rc0, u0, v0, sw0, st0 = batch_scale(ctx, mats, ps, plan=GROUP_PLAN)
    for plan in ([(16, "group", 1, 1), (32, "group", 1, 2), (48, "group", 2, 1), (64, "group", 2, 2),
                  (128, "group", 4, 2), (512, "block", 0, 0)],
                 [(32, "group", 1, 8), (64, "group", 2, 4), (128, "group", 4, 1), (512, "block", 0, 0)]):
        rc1, u1, v1, sw1, st1 = batch_scale(ctx, mats, ps, plan=plan)
        assert rc0 == 0 and rc1 == 0
        for a, b, c, d in zip(u0, v0, u1, v1):
            assert np.array_equal(a, c) and np.array_equal(b, d)
        assert np.array_equal(sw0, sw1)


def test_batch_rejects_large_n(ctx):
    rc, *_ = batch_scale(ctx, [W.uniform(600, 1, 1000, 3, dtype=np.int16)], [1.0])
    assert rc == L.SA_E_UNSUPPORTED
