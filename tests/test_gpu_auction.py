"""The reduced instance B solved with GPU-auction prices first (sa_solve_reduced_gpu).

The result must be the exact optimum (equal integer products with the oracle's dense
Hungarian method) with valid LP duals, like the host solver alone; the auction's own
assignment, when it completes within its round budget, must be within n * eps_final of
the optimum in sum of log weights (the eps-complementary-slackness bound of the auction)."""
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


def _csr(mask, w):
    rows, cols = np.nonzero(mask)
    rp = np.zeros(mask.shape[0] + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=mask.shape[0]), out=rp[1:])
    return rp, cols.astype(np.int32), w[rows, cols].astype(np.int32)


@pytest.mark.parametrize("n,density,hi,warm", [(1, 1.0, 5, False), (7, 1.0, 1000, False), (40, 0.15, 1000, False),
                                               (200, 0.05, 30000, True), (300, 1.0, 1000, False),
                                               (150, 0.3, 2, False), (120, 0.01, 3, True), (600, 0.1, 1000, True)])
def test_exact_optimum_and_auction_bound(ctx, n, density, hi, warm):
    rng = np.random.default_rng(n * 11 + hi)
    w = rng.integers(1, hi + 1, size=(n, n)).astype(np.int64)
    mask = rng.random((n, n)) < density
    mask[np.arange(n), rng.permutation(n)] = True
    rp, col, wv = _csr(mask, w)
    b = np.where(mask, np.log(w.astype(float)), -np.inf)
    price0 = None
    if warm:   # approximate duals, as the scaling provides: column maxima
        price0 = np.max(np.where(mask, b, -1e300), axis=0) * 0.5
    perm, s, al, be, info = api.sa_solve_reduced_gpu(ctx, rp, col, wv, price0=price0)
    assert sorted(perm) == list(range(n)) and all(mask[i, perm[i]] for i in range(n))
    ph, _, _, st = oracle.hungarian(b)
    assert st == 0
    assert oracle.perm_weight_exact(w, perm) == oracle.perm_weight_exact(w, ph)
    assert oracle.dual_violations(b, al, be, 1e-9)[0] == 0
    assert max(abs(al[i] + be[perm[i]] - b[i, perm[i]]) for i in range(n)) < 1e-9
    opt = sum(b[i, ph[i]] for i in range(n))
    assert abs(s - opt) < 1e-9
    if info["complete"]:
        assert info["auction_sum_log_w"] >= opt - n * info["eps_final"] - 1e-9, (info, opt)


@pytest.mark.parametrize("n,seed", [(12, 1), (30, 2)])
def test_auction_completes_within_eps_of_optimum(ctx, n, seed):
    """Small dense instances: the auction itself finishes every eps-scaling phase within
    its round budget, and its assignment is within n * eps_final of the optimum."""
    rng = np.random.default_rng(900 + seed)
    w = rng.integers(1, 1001, size=(n, n)).astype(np.int64)
    mask = np.ones((n, n), dtype=bool)
    rp, col, wv = _csr(mask, w)
    b = np.log(w.astype(float))
    perm, s, al, be, info = api.sa_solve_reduced_gpu(ctx, rp, col, wv)
    ph, _, _, st = oracle.hungarian(b)
    opt = sum(b[i, ph[i]] for i in range(n))
    assert info["complete"] == 1, info
    assert opt - n * info["eps_final"] - 1e-9 <= info["auction_sum_log_w"] <= opt + 1e-9
    assert abs(s - opt) < 1e-9


def test_reduced_instance_of_a_scaled_matrix(ctx):
    """B from the scaling and prune of a uniform n = 1024 matrix, warm prices v/p."""
    n = 1024
    w = W.uniform(n, 1, 1000, 1701, dtype=np.int16)
    d = api.to_device(w)
    ps = [1.0, 2.0, 4.0, 8.0]
    u, v, info = api.sa_scale(ctx, d, ps, 1e-6, 20000)
    rp, col, wv, _ = api.sa_prune(ctx, d, ps[-1], u, v)
    price0 = v.cpu().numpy() / ps[-1]
    perm_h, s_h, _, _ = api.sa_solve_reduced(rp, col, wv)
    perm_g, s_g, al, be, ai = api.sa_solve_reduced_gpu(ctx, rp, col, wv, price0=price0)
    assert abs(s_g - s_h) < 1e-9
    assert oracle.perm_weight_exact(w.astype(np.int64), perm_g) == oracle.perm_weight_exact(w.astype(np.int64), perm_h)
    assert ai["rounds"] >= 1
    # every search on the GPU runs at least one batch of 8 label-correcting rounds and one of
    # 8 tree levels
    assert ai["searches"] >= 0 and ai["search_rounds"] >= 16 * ai["searches"]


def test_no_perfect_matching(ctx):
    n = 50
    mask = np.zeros((n, n), dtype=bool)
    mask[:, :n - 1] = True            # column n-1 has no entry
    w = np.full((n, n), 5, dtype=np.int64)
    rp, col, wv = _csr(mask, w)
    with pytest.raises(api.SaError) as e:
        api.sa_solve_reduced_gpu(ctx, rp, col, wv)
    assert e.value.status == -5


def test_assign_through_gpu_auction_matches(ctx):
    """sa_assign with the context option SA_OPT_SOLVE_GPU = 1 returns the same certified
    optimum (at p = 1 about half of the entries pass t = 1/n, so B is above the GPU path's
    150000-entry threshold)."""
    n = 1000
    w = W.uniform(n, 1, 1000, 1702, dtype=np.int16)
    d = api.to_device(w)
    ps = [1.0]
    r1 = api.sa_assign(ctx, d, ps, 1e-6, 20000)
    c2 = api.sa_create(0)
    try:
        api.sa_set_option(c2, "solve_gpu", 1)
        r2 = api.sa_assign(c2, d, ps, 1e-6, 20000)
    finally:
        c2.close()
    assert r1["nnz_first"] >= 150000
    assert oracle.perm_weight_exact(w.astype(np.int64), r1["perm"]) == \
        oracle.perm_weight_exact(w.astype(np.int64), r2["perm"])


@pytest.mark.parametrize("n,hi,density", [(256, 1, 1.0), (400, 2, 0.2), (333, 1000, 0.05)])
def test_exact_dual_start_and_full_ties(ctx, n, hi, density):
    """The searches on the GPU at their degenerate extreme: prices started at an optimal dual
    (the oracle's beta), so every shortest augmenting path has length 0 and whole regions of
    columns sit at the same distance; with hi = 1 every entry ties.  The predecessor tree must
    stay acyclic and reach a free column behind columns at exactly that distance."""
    rng = np.random.default_rng(5000 + n + hi)
    w = rng.integers(1, hi + 1, size=(n, n)).astype(np.int64)
    mask = rng.random((n, n)) < density
    mask[np.arange(n), rng.permutation(n)] = True
    rp, col, wv = _csr(mask, w)
    b = np.where(mask, np.log(w.astype(float)), -np.inf)
    ph, _, beta, st = oracle.hungarian(b)
    assert st == 0
    for price0 in (beta, None):
        perm, s, al, be, _ = api.sa_solve_reduced_gpu(ctx, rp, col, wv, price0=price0)
        assert sorted(perm) == list(range(n)) and all(mask[i, perm[i]] for i in range(n))
        assert oracle.perm_weight_exact(w, perm) == oracle.perm_weight_exact(w, ph)
        assert oracle.dual_violations(b, al, be, 1e-9)[0] == 0
        assert max(abs(al[i] + be[perm[i]] - b[i, perm[i]]) for i in range(n)) < 1e-9
