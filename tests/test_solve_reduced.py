"""Host exact solver of the reduced instance (sa_solve_reduced) against the oracle's
dense Hungarian method: equal optimal products (exact integers) and valid LP duals.
Runs on the CPU: the solver is host code behind the C ABI."""
import numpy as np
import pytest

import oracle
from paper_1104_3830_gb300 import api


def _csr(mask, w):
    rows, cols = np.nonzero(mask)
    rp = np.zeros(mask.shape[0] + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=mask.shape[0]), out=rp[1:])
    return rp, cols.astype(np.int32), w[rows, cols].astype(np.int32)


@pytest.mark.parametrize("n,density,hi", [(1, 1.0, 5), (2, 1.0, 9), (7, 1.0, 1000), (40, 0.15, 1000),
                                          (200, 0.05, 30000), (300, 1.0, 1000), (257, 0.02, 7),
                                          # many ties (the row reduction's tie rule) and a single
                                          # allowed entry per row beside the permutation
                                          (150, 0.3, 2), (120, 0.01, 3), (400, 0.5, 4)])
def test_matches_oracle(n, density, hi):
    rng = np.random.default_rng(n * 7 + hi)
    w = rng.integers(1, hi + 1, size=(n, n)).astype(np.int64)
    mask = rng.random((n, n)) < density
    mask[np.arange(n), rng.permutation(n)] = True
    rp, col, wv = _csr(mask, w)
    perm, s, al, be = api.sa_solve_reduced(rp, col, wv)
    assert sorted(perm) == list(range(n)) and all(mask[i, perm[i]] for i in range(n))
    b = np.where(mask, np.log(w.astype(float)), -np.inf)
    ph, _, _, st = oracle.hungarian(b)
    assert st == 0
    assert oracle.perm_weight_exact(w, perm) == oracle.perm_weight_exact(w, ph)
    # duals: feasible on B, tight on the assignment
    assert oracle.dual_violations(b, al, be, 1e-9)[0] == 0
    assert max(abs(al[i] + be[perm[i]] - b[i, perm[i]]) for i in range(n)) < 1e-9
    assert abs(s - sum(b[i, perm[i]] for i in range(n))) < 1e-9


def test_no_perfect_matching_is_reported():
    # two rows that can only use the same column
    w = np.ones((3, 3), dtype=np.int64)
    mask = np.array([[1, 0, 0], [1, 0, 0], [1, 1, 1]], dtype=bool)
    rp, col, wv = _csr(mask, w)
    with pytest.raises(api.SaError) as e:
        api.sa_solve_reduced(rp, col, wv)
    assert e.value.status == -5


def _check(mask, w, perm, s, al, be):
    n = len(perm)
    assert sorted(perm) == list(range(n)) and all(mask[i, perm[i]] for i in range(n))
    b = np.where(mask, np.log(w.astype(float)), -np.inf)
    ph, _, _, st = oracle.hungarian(b)
    assert st == 0
    assert oracle.perm_weight_exact(w, perm) == oracle.perm_weight_exact(w, ph)
    assert oracle.dual_violations(b, al, be, 1e-9)[0] == 0
    assert max(abs(al[i] + be[perm[i]] - b[i, perm[i]]) for i in range(n)) < 1e-9
    assert abs(s - sum(b[i, perm[i]] for i in range(n))) < 1e-9


@pytest.mark.parametrize("n,density,hi,start", [(60, 0.2, 1000, "exact"), (150, 0.3, 2, "exact"),
                                                (200, 0.05, 30000, "noisy"), (300, 1.0, 1, "noisy"),
                                                (257, 0.02, 7, "exact"), (400, 0.5, 4, "noisy"),
                                                (90, 0.1, 1000, "nonfinite")])
def test_warm_start_matches_oracle(n, density, hi, start):
    """sa_solve_reduced_warm from given column duals: the exact duals of the instance itself
    (every search then has length 0, the most tied case), the same plus noise (approximate
    duals, as the scaling gives), or duals with non-finite entries (the column minimum is
    used there).  The optimum and the LP duals are exact whatever the start."""
    rng = np.random.default_rng(n * 13 + hi)
    w = rng.integers(1, hi + 1, size=(n, n)).astype(np.int64)
    mask = rng.random((n, n)) < density
    mask[np.arange(n), rng.permutation(n)] = True
    rp, col, wv = _csr(mask, w)
    b = np.where(mask, np.log(w.astype(float)), -np.inf)
    _, _, beta_opt, st = oracle.hungarian(b)
    assert st == 0
    beta0 = beta_opt.copy()
    if start == "noisy":
        beta0 += rng.normal(0.0, 0.05, size=n)
    elif start == "nonfinite":
        beta0[::3] = np.nan
        beta0[1::7] = np.inf
    perm, s, al, be = api.sa_solve_reduced(rp, col, wv, beta0=beta0)
    _check(mask, w, perm, s, al, be)


def test_warm_start_argument_checks():
    rp, col, wv = _csr(np.eye(3, dtype=bool), np.full((3, 3), 2, dtype=np.int64))
    with pytest.raises(ValueError):
        api.sa_solve_reduced(rp, col, wv, beta0=np.zeros(2))
    perm, s, _, _ = api.sa_solve_reduced(rp, col, wv, beta0=np.zeros(3))
    assert list(perm) == [0, 1, 2] and abs(s - 3 * np.log(2.0)) < 1e-12


def test_early_stop_on_ties_at_the_free_column():
    """Every entry equal (all reduced costs 0 from the column minima): each search reaches a
    free column at distance 0 and stops there; the result is still a permutation of B with
    exact duals."""
    n = 500
    rng = np.random.default_rng(4)
    mask = rng.random((n, n)) < 0.05
    mask[np.arange(n), rng.permutation(n)] = True
    w = np.full((n, n), 7, dtype=np.int64)
    rp, col, wv = _csr(mask, w)
    perm, s, al, be = api.sa_solve_reduced(rp, col, wv)
    _check(mask, w, perm, s, al, be)


@pytest.mark.parametrize("n,density,hi,shift", [(60, 0.2, 1000, 0.0), (150, 0.3, 2, 0.3), (200, 0.05, 30000, -0.2),
                                                (300, 1.0, 1, 0.0), (257, 0.02, 7, 1.0), (1, 1.0, 5, 0.0)])
def test_near_duals_are_the_largest_below_the_target(n, density, hi, shift):
    """sa_solve_reduced_near: the optimum of B with LP-optimal duals whose beta is the
    componentwise largest with beta <= near.  Checked by the characterisation of that
    largest solution of the difference constraints: optimal and feasible on B, beta <= near,
    and every column below its target is held down by a tight entry (an entry (i, j) of
    B whose constraint beta_{perm(i)} <= beta_j + log w_{i perm(i)} - log w_ij is an
    equality)."""
    rng = np.random.default_rng(n * 17 + hi)
    w = rng.integers(1, hi + 1, size=(n, n)).astype(np.int64)
    mask = rng.random((n, n)) < density
    mask[np.arange(n), rng.permutation(n)] = True
    rp, col, wv = _csr(mask, w)
    b = np.where(mask, np.log(w.astype(float)), -np.inf)
    _, _, beta_opt, _ = oracle.hungarian(b)
    near = beta_opt + shift + rng.normal(0.0, 0.05, size=n)
    perm, s, al, be = api.sa_solve_reduced(rp, col, wv, near=near)
    _check(mask, w, perm, s, al, be)
    assert np.all(be <= near + 1e-12)
    rows, cols = np.nonzero(mask)
    for k in range(n):
        if be[k] >= near[k] - 1e-9:
            continue
        i_k = int(np.nonzero(perm == k)[0][0])
        js = cols[rows == i_k]
        gaps = [be[j] + b[i_k, k] - b[i_k, j] - be[k] for j in js if j != k]
        # the column's dual is held down by a tight constraint through its row
        assert gaps and min(gaps) < 1e-9, (k, gaps)


def test_near_with_optimal_target_returns_it():
    """A target that is itself an optimal dual of B comes back unchanged (the largest
    optimal beta below it is itself)."""
    rng = np.random.default_rng(99)
    n = 120
    w = rng.integers(1, 1001, size=(n, n)).astype(np.int64)
    mask = rng.random((n, n)) < 0.1
    mask[np.arange(n), rng.permutation(n)] = True
    rp, col, wv = _csr(mask, w)
    b = np.where(mask, np.log(w.astype(float)), -np.inf)
    _, _, beta_opt, _ = oracle.hungarian(b)
    perm, s, al, be = api.sa_solve_reduced(rp, col, wv, near=beta_opt)
    _check(mask, w, perm, s, al, be)
    assert np.max(np.abs(be - beta_opt)) < 1e-9


@pytest.mark.parametrize("case", ["uniform", "zipf", "planted", "tied", "few_values"])
def test_near_duals_certify_all_of_a(case):
    """The first solve of sa_assign on the host: B from the oracle's scaling and prune
    (t = 1/n), solved by sa_solve_reduced_near toward v/p.  On these seeded workloads the
    returned duals hold on all of A (no entry for the certificate to add), while the duals
    of the plain solve from the column minima miss entries on the Zipf workload."""
    from paper_1104_3830_gb300 import workloads as W
    ps = [2.0 ** k for k in range(9)]
    if case == "uniform":
        w = W.uniform(160, 1, 1000, 31, dtype=np.int32)
    elif case == "zipf":
        w = W.zipf(300, 1.2, 30000, 603)
    elif case == "planted":
        w, _, _ = W.planted(200, 32)
    elif case == "tied":
        w, _, _ = W.planted(256, 33, tied_frac=0.05)
    else:
        w = W.uniform(150, 1, 3, 34, dtype=np.int32)
    w = np.asarray(w).astype(np.int64)
    b = oracle.log_weights(w)
    u, v, _, _, _ = oracle.sinkhorn(b, ps, 1e-6, 2000)
    m = oracle.prune_mask(b, ps[-1], u, v)
    rp, col = oracle.prune_csr(m)
    wv = w[m].astype(np.int32)
    perm, s, al, be = api.sa_solve_reduced(rp, col, wv, near=v / ps[-1])
    assert all(m[i, perm[i]] for i in range(len(perm)))
    assert oracle.dual_violations(b, al, be, 1e-9)[0] == 0
    assert oracle.perm_weight_exact(w, perm) == oracle.perm_weight_exact(w, oracle.hungarian(b)[0])
    if case == "zipf":
        _, _, alc, bec = api.sa_solve_reduced(rp, col, wv)
        assert oracle.dual_violations(b, alc, bec, 1e-9)[0] > 0


def test_repeated_columns_in_a_row():
    """A caller's CSR may list a column twice in a row with different weights: the solvers
    then use the larger weight, and the near duals stay feasible on every listed entry."""
    rp = np.array([0, 3, 5, 7], dtype=np.int64)
    col = np.array([0, 0, 1, 1, 2, 2, 0], dtype=np.int32)
    w = np.array([2, 9, 3, 5, 1, 4, 7], dtype=np.int32)
    for kw in ({}, {"near": np.zeros(3)}, {"beta0": np.ones(3)}):
        perm, s, al, be = api.sa_solve_reduced(rp, col, w, **kw)
        assert sorted(perm) == [0, 1, 2]
        lw = np.log(w.astype(float))
        rows = np.repeat(np.arange(3), np.diff(rp))
        assert np.all(al[rows] + be[col] >= lw - 1e-12)
        # the best permutation: row0 -> col0 (9), row1 -> col1 (5), row2 -> col2 (4)
        assert list(perm) == [0, 1, 2] and abs(s - np.log(9 * 5 * 4)) < 1e-12
