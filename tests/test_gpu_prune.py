"""Parity of pruning / compaction (sa_prune), the certificate of Prop. aoc, the duality
check (sa_certify) and the whole pipeline (sa_assign) with the oracle.

Prune decisions are compared bit for bit on the same FP64 potentials (the oracle's),
except entries whose FP64 log-domain value lies within 1e-9 of log t, where the last bit
of two different FP64 logarithms may decide.  The final assignment must have the same
exact integer product as the oracle's dense Hungarian optimum."""
import numpy as np
import pytest

import oracle
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


def _oracle_case(n, seed, ps, dtype=np.int32, hi=1000):
    w = W.uniform(n, 1, hi, seed, dtype=dtype)
    b = oracle.log_weights(w.astype(np.int64))
    u, v, *_ = oracle.sinkhorn(b, ps, 1e-8, 20000)
    return w, b, u, v


@pytest.mark.parametrize("n,dtype,guard,t", [(256, np.int32, True, 0.0), (300, np.int16, False, 0.0),
                                             (1001, np.int16, True, 0.0), (64, np.int32, True, 0.5),
                                             (5, np.int16, True, 0.0)])
def test_prune_matches_oracle(ctx, n, dtype, guard, t):
    ps = [1.0, 2.0, 4.0, 8.0, 16.0]
    w, b, u, v = _oracle_case(n, 300 + n, ps, dtype)
    d = api.to_device(w)
    rp, col, wv, ub = api.sa_prune(ctx, d, ps[-1], torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), t, guard)
    mask_g = np.zeros((n, n), dtype=bool)
    rows = np.repeat(np.arange(n), np.diff(rp))
    mask_g[rows, col] = True
    assert np.all(np.diff(col[rp[:-1].clip(max=len(col) - 1)]) >= -n)  # well formed
    for i in range(n):
        assert np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0)
    assert np.array_equal(wv, w[rows, col])
    tt = t if t > 0 else 1.0 / n
    mask_o = oracle.prune_mask(b, ps[-1], u, v, tt, guard)
    e = ps[-1] * b - u[:, None] - v[None, :]
    near = np.abs(e - np.log(tt)) < 1e-9
    assert np.array_equal(mask_g & ~near, mask_o & ~near)
    if guard:
        assert mask_g.any(axis=1).all() and mask_g.any(axis=0).all()
    assert abs(ub - oracle.log_ub(b, ps[-1], v)) < 1e-9 * max(1.0, abs(ub))


def test_certify_counts_like_oracle(ctx):
    w = W.uniform(200, 1, 1000, 500, dtype=np.int16)
    b = oracle.log_weights(w.astype(np.int64))
    perm, al, be, _ = oracle.hungarian(b)
    d = api.to_device(w)
    nv, _ = api.sa_certify(ctx, d, al, be, 1e-9)
    assert nv == 0
    bb = b.copy()
    bb[np.arange(200), perm] = -np.inf
    _, al2, be2, _ = oracle.hungarian(bb)
    nv2, (rp, col, wv) = api.sa_certify(ctx, d, al2, be2, 1e-9)
    cnt, _ = oracle.dual_violations(b, al2, be2, 1e-9)
    assert nv2 == cnt and rp[-1] == cnt
    rows = np.repeat(np.arange(200), np.diff(rp))
    assert np.all(b[rows, col] - al2[rows] - be2[col] > 1e-9)
    assert np.array_equal(wv, w[rows, col])


@pytest.mark.parametrize("case", ["c1", "uniform777", "planted2048", "tied1024", "zipf300"])
def test_assign_is_exactly_optimal(ctx, case):
    if case == "c1":
        w, ps = W.c1()
    elif case == "uniform777":
        w, ps = W.uniform(777, 1, 1000, 600, dtype=np.int16), [2.0 ** k for k in range(8)]
    elif case == "planted2048":
        w, pi, _ = W.planted(2048, 601)
        ps = [2.0 ** k for k in range(10)]
    elif case == "tied1024":
        w, pi, _ = W.planted(1024, 602, tied_frac=0.01)
        ps = [2.0 ** k for k in range(10)]
    else:
        w, ps = W.zipf(300, 1.2, 30000, 603), [2.0 ** k for k in range(9)]
    d = api.to_device(w)
    r = api.sa_assign(ctx, d, ps, 1e-6, 2000)
    perm = r["perm"]
    assert sorted(perm) == list(range(len(perm)))
    b = oracle.log_weights(w.astype(np.int64))
    if case.startswith("planted") or case.startswith("tied"):
        ref = oracle.perm_weight_exact(w, pi)
    else:
        ref = oracle.perm_weight_exact(w, oracle.hungarian(b)[0])
    assert oracle.perm_weight_exact(w, perm) == ref
    assert r["gamma"] >= 1 - 1e-9
    assert r["nnz_first"] < w.size


def test_assign_host_equals_device(ctx):
    w, ps = W.c1()
    d = api.to_device(w)
    r1 = api.sa_assign(ctx, d, ps)
    r2 = api.sa_assign_host(ctx, w, ps)
    assert oracle.perm_weight_exact(w, r1["perm"]) == oracle.perm_weight_exact(w, r2["perm"])
    assert r1["scale"]["sweeps_total"] == r2["scale"]["sweeps_total"]


def test_narrowing(ctx):
    w = W.uniform(100, 1, 32767, 700, dtype=np.int32)
    src = torch.from_numpy(w).cuda()
    dst = torch.zeros((100, 104), dtype=torch.int16, device="cuda")[:, :100]
    assert api.sa_narrow_i32_to_i16(ctx, src, dst) == 0
    assert np.array_equal(dst.cpu().numpy().astype(np.int32), w)
    src[3, 4] = 40000
    assert api.sa_narrow_i32_to_i16(ctx, src, dst) == 1
