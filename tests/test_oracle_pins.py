"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics, not to itself.

Each test names the passage it follows.  Together they are chosen so that a dropped
term, a sign or index slip or a transposed operand anywhere in the oracle fails one of
them: the 3x3 example is not symmetric (catches transposition), the closed forms fix
exact values (catch dropped terms and signs), the solvers are checked against each
other, scipy and exhaustive search.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_1104_3830_gb300 import workloads as W


def _bist(b, p, tol=1e-12, sweeps=200000, loose=None):
    """X(p) by the oracle; with loose set, accept a capped run whose residual is below it
    (nearly decomposable A(p) converge sublinearly, Sec. 3.1)."""
    u, v, sw, rs, st = oracle.sinkhorn(b, [p], tol, sweeps)
    assert st == 0 or (loose is not None and rs[0] < loose)
    return oracle.xmatrix(b, p, u, v), u, v


# --- P1: the worked 3x3 example (Sec. 2.3) -------------------------------------------
def test_example_3x3_matches_printed_x10(golden):
    g = golden("example_3x3.txt")
    a = np.array(g["A"])
    a[1, 2] = 1.0 / 3.0
    x, _, _ = _bist(oracle.log_weights(a), g["p"])
    want = np.array(g["X"])
    assert np.max(np.abs(x - want)) < 1e-4
    # the transposed problem gives the transposed matrix, which is far from the print
    xt, _, _ = _bist(oracle.log_weights(a.T), g["p"])
    assert np.max(np.abs(xt - want)) > 1e-2
    assert np.allclose(xt, x.T, atol=1e-9)


def test_example_3x3_certificate_is_tight():
    # row maxima of A lie on the identity, the optimal permutation, so the bound of
    # Prop. aoc is >= log w_opt(A) = 0 for any potentials and equals it once X(p) is
    # dominated by the identity (p = 2000 converges in one sweep)
    a = np.array([[1, 0.99, 0.99], [0.99, 1, 1 / 3], [0.25, 0.5, 1]])
    b = oracle.log_weights(a)
    for p in (10.0, 50.0, 400.0):
        u, v, *_ = oracle.sinkhorn(b, [p], 1e-8, 200)
        assert oracle.log_ub(b, p, v) >= -1e-12
    _, _, v = _bist(b, 2000.0, tol=1e-8)
    assert abs(oracle.log_ub(b, 2000.0, v)) < 1e-9


# --- P2: the 5x5 example (Sec. 4.2) --------------------------------------------------
def test_example_5x5_optimal_permutation(golden):
    g = golden("example_5x5.txt")
    a = np.array(g["A"])
    want = [int(k) - 1 for k in g["perm"][0]]
    b = oracle.log_weights(a)
    assert list(oracle.hungarian(b)[0]) == want
    assert list(oracle.lapjv(b)[0]) == want
    assert list(oracle.bruteforce(b)[0]) == want
    x, _, _ = _bist(b, g["p"], tol=1e-10, sweeps=20000, loose=1e-3)
    assert list(np.argmax(x, axis=1)) == want
    assert list(np.argmax(x, axis=0)) == list(np.argsort(want))
    # the optimal entries dominate: (1 +- O(e^{-cp})) vs O(e^{-cp}) (Sec. 4.2)
    assert min(x[i, want[i]] for i in range(5)) > 0.9


# --- P3: 2x2 closed form; Cor. exponential_conv ---------------------------------------
@pytest.mark.parametrize("seed", range(5))
def test_2x2_closed_form(seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.1, 3.0, size=(2, 2))
    b = oracle.log_weights(a)
    for p in (0.5, 1.0, 3.0, 10.0):
        x, _, _ = _bist(b, p, tol=1e-13)
        k = (a[0, 0] * a[1, 1] / (a[0, 1] * a[1, 0])) ** p
        s = math.sqrt(k) / (1 + math.sqrt(k))
        assert np.allclose(x, [[s, 1 - s], [1 - s, s]], atol=1e-12, rtol=0)


def test_exponential_rate_2x2():
    # 1 - x_11(p) = 1/(1 + sqrt(K)) with K = cross-ratio^p: log distance is linear in p
    # with slope -log(cross ratio)/2 (Cor. exponential_conv with an explicit c)
    a = np.array([[2.0, 1.0], [1.0, 1.5]])
    b = oracle.log_weights(a)
    ps = np.array([8.0, 10.0, 12.0, 14.0])
    d = []
    for p in ps:
        x, _, _ = _bist(b, p, tol=1e-14)
        d.append(math.log(x[0, 1]))
    slope = np.polyfit(ps, d, 1)[0]
    assert abs(slope + 0.5 * math.log(3.0)) < 1e-2


# --- P4: rank one matrices scale to J/n (Thm. prop-borweinlewisnussbaum) ------------
def test_rank_one_gives_uniform():
    rng = np.random.default_rng(3)
    r, c = rng.uniform(0.5, 5, 7), rng.uniform(0.5, 5, 7)
    b = oracle.log_weights(np.outer(r, c))
    for p in (1.0, 7.0, 100.0):
        x, _, _ = _bist(b, p)
        assert np.allclose(x, 1 / 7, atol=1e-12)


# --- P5: invariances ---------------------------------------------------------------
def test_permutation_transpose_and_diagonal_invariance():
    rng = np.random.default_rng(4)
    a = rng.uniform(1, 100, size=(9, 9))
    p = 3.0
    x, _, _ = _bist(oracle.log_weights(a), p)
    pr, pc = rng.permutation(9), rng.permutation(9)
    xp, _, _ = _bist(oracle.log_weights(a[pr][:, pc]), p)
    assert np.allclose(xp, x[pr][:, pc], atol=1e-10)
    xt, _, _ = _bist(oracle.log_weights(a.T), p)
    assert np.allclose(xt, x.T, atol=1e-10)
    d1, d2 = rng.uniform(0.1, 10, 9), rng.uniform(0.1, 10, 9)
    xd, _, _ = _bist(oracle.log_weights(d1[:, None] * a * d2[None, :]), p)
    assert np.allclose(xd, x, atol=1e-10)


def test_prescaling_identity():
    # Sec. 4.1.1: prescaling maps A to A^(m)/c in [1, e]; X(A^(m)/c, q) = X(A, q*m)
    rng = np.random.default_rng(5)
    a = rng.integers(1, 1000, size=(8, 8)).astype(float)
    s, m, c = oracle.prescale(a)
    assert s.min() >= 1 - 1e-12 and s.max() <= math.e + 1e-12
    assert abs(m - 1 / math.log(a.max() / a.min())) < 1e-15
    for q in (10.0, 50.0):
        x1, _, _ = _bist(oracle.log_weights(s), q)
        x2, _, _ = _bist(oracle.log_weights(a), q * m)
        assert np.allclose(x1, x2, atol=1e-9)
    # prescaling makes A^(k) and A land on the same matrix (invariance under powers)
    s2, _, _ = oracle.prescale(a ** 3)
    assert np.allclose(s, s2, atol=1e-12)


# --- P6 / P10: exact solvers --------------------------------------------------------
@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 8])
def test_solvers_agree_with_bruteforce(n):
    from scipy.optimize import linear_sum_assignment
    rng = np.random.default_rng(100 + n)
    for trial in range(6):
        w = rng.integers(1, 30 if trial % 2 else 1000, size=(n, n))
        b = oracle.log_weights(w)
        exact = max(math.prod(int(w[i, s[i]]) for i in range(n))
                    for s in itertools.permutations(range(n)))
        ph, al, be, st = oracle.hungarian(b)
        pj, _ = oracle.lapjv(b)
        pb, best, _ = oracle.bruteforce(b)
        _, cs = linear_sum_assignment(-b)
        for perm in (ph, pj, pb, cs):
            assert sorted(perm) == list(range(n))
            assert oracle.perm_weight_exact(w, perm) == exact
        assert oracle.dual_violations(b, al, be, 1e-9)[0] == 0
        assert all(abs(al[i] + be[ph[i]] - b[i, ph[i]]) < 1e-9 for i in range(n))


def test_solvers_agree_larger_and_with_forbidden_entries():
    from scipy.optimize import linear_sum_assignment
    rng = np.random.default_rng(7)
    for n in (40, 120):
        w = rng.integers(1, 1000, size=(n, n))
        b = oracle.log_weights(w)
        ph = oracle.hungarian(b)[0]
        pj = oracle.lapjv(b)[0]
        _, cs = linear_sum_assignment(-b)
        ref = oracle.perm_weight_exact(w, cs)
        assert oracle.perm_weight_exact(w, ph) == ref
        assert oracle.perm_weight_exact(w, pj) == ref
        # sparse pattern that still holds a permutation: forbidden entries handled
        mask = rng.random((n, n)) < 0.1
        mask[np.arange(n), rng.permutation(n)] = True
        wb = np.where(mask, w, 0)
        bb = oracle.log_weights(wb)
        ph2, al, be, st = oracle.hungarian(bb)
        assert st == 0 and all(mask[i, ph2[i]] for i in range(n))
        big = 10.0 ** 9
        _, cs2 = linear_sum_assignment(np.where(mask, -b, big))
        assert oracle.perm_weight_exact(wb, ph2) == oracle.perm_weight_exact(wb, cs2)
    # no perfect matching: a zero row
    w = np.ones((4, 4))
    w[2] = 0
    assert oracle.hungarian(oracle.log_weights(w))[3] == oracle.E_INFEASIBLE


def test_dual_violation_detects_missing_entry():
    rng = np.random.default_rng(8)
    w = rng.integers(1, 1000, size=(30, 30))
    b = oracle.log_weights(w)
    perm, al, be, _ = oracle.hungarian(b)
    assert oracle.dual_violations(b, al, be, 1e-9)[0] == 0
    # duals of a sub-problem that lost the optimum's entries are infeasible on A
    bb = b.copy()
    bb[np.arange(30), perm] = -np.inf
    p2, al2, be2, st = oracle.hungarian(bb)
    assert st == 0
    cnt, gap = oracle.dual_violations(b, al2, be2, 1e-9)
    assert cnt > 0 and gap > 0


# --- Prop. aoc: the certificate bounds the optimum for any potentials ----------------
def test_certificate_upper_bound_any_v_and_gamma():
    rng = np.random.default_rng(9)
    for n in (4, 6, 8):
        w = rng.integers(1, 1000, size=(n, n))
        b = oracle.log_weights(w)
        opt = oracle.bruteforce(b)[1]
        for p in (1.0, 5.0, 40.0):
            for _ in range(3):
                v = rng.normal(0, 10, n)
                assert oracle.log_ub(b, p, v) >= opt - 1e-12
            r = oracle.preprocess(w, [p], tol=1e-9)
            assert r["log_ub"] >= opt - 1e-9
            assert r["gamma"] >= 1 - 1e-9


# --- P7 / P8: convergence to the optimal face (Thm. prop-converge1) ------------------
def test_planted_converges_to_permutation():
    w, pi, _ = W.planted(48, 11)
    b = oracle.log_weights(w.astype(np.int64))
    assert list(oracle.hungarian(b)[0]) == list(pi)
    ps = [8.0, 16.0, 32.0, 64.0, 128.0]
    dist = []
    for p in ps:
        x, _, _ = _bist(b, p, tol=1e-11, sweeps=20000, loose=1e-3)
        perm_mat = np.zeros_like(x)
        perm_mat[np.arange(48), pi] = 1
        dist.append(np.max(np.abs(x - perm_mat)))
    assert all(d2 < d1 for d1, d2 in zip(dist, dist[1:]))
    assert dist[-1] < 1e-2
    # O(exp(-cp)) (Cor. exponential_conv): log distance falls at least linearly in p
    slope = np.polyfit(ps[-3:], np.log(dist[-3:]), 1)[0]
    assert slope < -0.01


def test_tied_planted_limit_is_max_entropy_face():
    w, pi, pairs = W.planted(40, 12, tied_frac=0.2)
    assert len(pairs) == 4
    b = oracle.log_weights(w.astype(np.int64))
    x, _, _ = _bist(b, 600.0, tol=1e-12, sweeps=20000, loose=1e-3)
    want = np.zeros((40, 40))
    want[np.arange(40), pi] = 1.0
    for i, k in pairs:
        for r in (i, k):
            for c in (pi[i], pi[k]):
                want[r, c] = 0.5
    assert np.max(np.abs(x - want)) < 1e-3


# --- P9: bistochastic, and independence of the path (uniqueness of X(p)) -------------
def test_bistochastic_and_warm_start_independent():
    w = W.uniform(64, 1, 1000, 13)
    b = oracle.log_weights(w)
    ps = [1.0, 2.0, 4.0, 8.0, 16.0]
    u1, v1, _, rs, st = oracle.sinkhorn(b, ps, 1e-11, 100000)
    assert st == 0 and rs[-1] <= 1e-11
    r, c = oracle.sums(b, ps[-1], u1, v1)
    assert np.max(np.abs(r - 1)) < 1e-9 and np.max(np.abs(c - 1)) < 1e-9
    u2, v2, _, _, st2 = oracle.sinkhorn(b, ps, 1e-11, 100000, warm_keep_v=True)
    assert st2 == 0
    x1 = oracle.xmatrix(b, 16.0, u1, v1)
    x2 = oracle.xmatrix(b, 16.0, u2, v2)
    assert np.max(np.abs(x1 - x2)) < 1e-9
    # starting from arbitrary potentials lands on the same X(p)
    u3, v3, _, _, st3 = oracle.sinkhorn_from(b, 16.0, np.zeros(64), np.random.default_rng(1).normal(0, 3, 64), 1e-11, 100000)
    assert st3 == 0
    assert np.max(np.abs(oracle.xmatrix(b, 16.0, u3, v3) - x1)) < 1e-9


def test_not_converged_status_and_no_support():
    w = W.uniform(32, 1, 1000, 14)
    b = oracle.log_weights(w)
    _, _, sw, _, st = oracle.sinkhorn(b, [64.0], 1e-12, 3)
    assert st == oracle.NOT_CONVERGED and sw[0] == 3
    w0 = w.copy()
    w0[5] = 0
    assert oracle.sinkhorn(oracle.log_weights(w0), [1.0], 1e-6, 10)[4] == oracle.E_NO_SUPPORT


# --- pruning (Eq. matrixred) --------------------------------------------------------
def test_prune_threshold_and_guard():
    w = W.uniform(50, 1, 1000, 15)
    b = oracle.log_weights(w)
    u, v, *_ = oracle.sinkhorn(b, [1.0, 2.0, 4.0, 8.0], 1e-9, 100000)
    x = oracle.xmatrix(b, 8.0, u, v)
    m = oracle.prune_mask(b, 8.0, u, v, guard=False)
    assert np.array_equal(m, x >= 1 / 50)
    mg = oracle.prune_mask(b, 8.0, u, v, t=0.9, guard=True)
    assert mg.any(axis=1).all() and mg.any(axis=0).all()
    assert np.array_equal(mg, (x >= 0.9) | (x == x.max(axis=1, keepdims=True)) | (x == x.max(axis=0, keepdims=True)))
    rp, col = oracle.prune_csr(m)
    assert rp[-1] == m.sum() and all(np.array_equal(np.nonzero(m[i])[0], col[rp[i]:rp[i + 1]]) for i in range(50))


# ---- Algorithm 1 with adaptive p (Sec. 4.2) -----------------------------------------

def test_algorithm1_gamma_bounds_the_brute_force_optimum():
    """On small instances the returned permutation of B is within the factor gamma of the
    optimum of A found by enumeration (Prop. aoc), and gamma <= opt_ratio on success."""
    for seed in range(4):
        w = W.uniform(7, 1, 50, 700 + seed, dtype=np.int32)
        r = oracle.algorithm1(w, opt_ratio=1.5, p0=5.0, dp=5.0, max_rounds=40, eps=1e-9)
        assert r["status"] == 0 and r["gamma"] <= 1.5
        b = oracle.log_weights(w.astype(np.int64))
        perm_bf, best = oracle.bruteforce(b)[:2]
        # the reported weight is the returned permutation's own, and it is within gamma of
        # the enumerated optimum
        assert abs(b[np.arange(7), r["perm"]].sum() - r["log_w_B"]) < 1e-9
        assert -1e-12 <= best - r["log_w_B"] <= np.log(r["gamma"]) + 1e-9
        assert sorted(r["perm"]) == list(range(7))


def test_algorithm1_planted_stops_in_one_round():
    """A planted strict row maximum: the first p already isolates the plant, and the certified
    ratio is within the requested bound (gamma tends to 1 only as p grows)."""
    w, pi, _ = W.planted(64, W.BASE_SEED + 90)
    r = oracle.algorithm1(w, opt_ratio=2.0)
    assert r["status"] == 0 and r["rounds"] == 1
    assert np.array_equal(r["perm"], pi)
    assert 1.0 <= r["gamma"] <= 2.0


def test_algorithm1_prescaling_scale():
    """p is on the prescaled scale: p_raw = p / ln(max/min) when max/min > e, p otherwise."""
    w = W.uniform(16, 1, 1000, 91, dtype=np.int32)
    r = oracle.algorithm1(w, opt_ratio=1e9, p0=100.0)
    ratio = w.max() / w[w > 0].min()
    assert abs(r["p_raw"] - 100.0 / np.log(ratio)) < 1e-12
    w2 = (np.ones((16, 16)) * 2 + np.eye(16)).astype(np.int32)   # max/min = 1.5 < e
    r2 = oracle.algorithm1(w2, opt_ratio=1e9, p0=100.0)
    assert r2["p_raw"] == 100.0


def test_thread_count_does_not_change_the_result():
    """The oracle's parallel loops split independent rows or columns, so one thread and all
    threads give bit-identical potentials (the one-core CPU baseline times the same
    arithmetic)."""
    w = W.uniform(97, 1, 1000, 4242, dtype=np.int32).astype(np.int64)
    b = oracle.log_weights(w)
    k = oracle.num_threads()
    u0, v0 = np.zeros(97), np.zeros(97)
    ua, va, *_ = oracle.sinkhorn_from(b, 4.0, u0, v0, 1e-300, 40)
    oracle.set_num_threads(1)
    try:
        ub, vb, *_ = oracle.sinkhorn_from(b, 4.0, u0, v0, 1e-300, 40)
    finally:
        oracle.set_num_threads(k)
    assert oracle.num_threads() == k
    assert np.array_equal(ua, ub) and np.array_equal(va, vb)
