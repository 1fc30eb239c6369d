"""Pins of the oracle's deformed Sinkhorn iteration (Sec. 3.2): one sweep at each p_m of an
increasing sequence with the column potentials v carried from one p to the next
(`oracle.sinkhorn(..., max_sweeps=1, warm_keep_v=True)`).

1. The paper defines the iteration multiplicatively (Eqs. colscale and rowscale):
   Z_0 = ROWS(A^(p_1)), W_m = COLS(Z_{m-1}), Z_m = ROWS(W_m o A^(p_{m+1} - p_m)).  That
   recursion is written out here on explicit matrices (entrywise powers and Hadamard
   products, no potentials, no logarithms) and W_M must equal the oracle's iterate after
   M sweeps, which it forms as exp(p_M b - u - v) from log-domain potentials.  Rescaling v
   by p_{m+1}/p_m between steps (the library's default warm start) is a different
   iteration, and the pin tells the two apart.
2. Theorem logconvergencepositive: for a positive A and p_m = a log(m + 1) with
   0 < a log theta(A) < 2 (theta of Sec. 3.1), the iteration converges to a bistochastic
   matrix whose mass lies on the optimal permutation.
"""
import itertools
import math

import numpy as np
import pytest

import oracle


def _rows(x):
    return x / x.sum(axis=1, keepdims=True)


def _cols(x):
    return x / x.sum(axis=0, keepdims=True)


def _paper_recursion(a_mat, ps):
    z = _rows(a_mat ** ps[0])
    for m in range(1, len(ps)):
        z = _rows(_cols(z) * a_mat ** (ps[m] - ps[m - 1]))
    return _cols(z)


def _theta(a_mat):
    n = a_mat.shape[0]
    return max(a_mat[i, r] * a_mat[j, l] / (a_mat[j, r] * a_mat[i, l])
               for i, j, r, l in itertools.product(range(n), repeat=4))


@pytest.mark.parametrize("n,a,steps,seed", [(5, 0.7, 60, 3), (7, 2.0, 40, 4), (3, 0.25, 200, 5)])
def test_iteration_equals_the_papers_recursion(n, a, steps, seed):
    rng = np.random.default_rng(seed)
    a_mat = rng.uniform(1.0, 3.0, size=(n, n))
    b = np.log(a_mat)
    ps = [a * math.log(m + 1) for m in range(1, steps + 1)]
    w_m = _paper_recursion(a_mat, ps)
    u, v, sw, _, _ = oracle.sinkhorn(b, ps, 1e-300, 1, warm_keep_v=True)
    assert int(sw.sum()) == steps
    x = oracle.xmatrix(b, ps[-1], u, v)
    assert np.max(np.abs(x - w_m)) < 1e-12
    # the default warm start (v rescaled with p) is another iteration: the pin sees it
    u2, v2, _, _, _ = oracle.sinkhorn(b, ps, 1e-300, 1, warm_keep_v=False)
    assert np.max(np.abs(oracle.xmatrix(b, ps[-1], u2, v2) - w_m)) > 1e-8


def test_converges_to_the_optimal_assignment():
    """Positive A with a unique optimal permutation and a log theta = 1.9: the row residual
    of the column-stochastic iterate shrinks as the sweeps go on, and the iterate gathers on
    the optimal permutation."""
    rng = np.random.default_rng(11)
    n = 6
    perm = rng.permutation(n)
    a_mat = rng.uniform(1.0, 1.5, size=(n, n))
    a_mat[np.arange(n), perm] = 2.0
    b = np.log(a_mat)
    best = oracle.bruteforce(b)[0]
    assert list(best) == list(perm)
    a = 1.9 / math.log(_theta(a_mat))
    out = []
    for steps in (1000, 10000):
        ps = [a * math.log(m + 1) for m in range(1, steps + 1)]
        u, v, _, _, _ = oracle.sinkhorn(b, ps, 1e-300, 1, warm_keep_v=True)
        x = oracle.xmatrix(b, ps[-1], u, v)
        assert np.max(np.abs(x.sum(axis=0) - 1.0)) < 1e-12      # the column update is last
        out.append((np.max(np.abs(x.sum(axis=1) - 1.0)), x[np.arange(n), perm].min()))
    (r1, m1), (r2, m2) = out
    assert r2 < r1 / 5 and r2 < 1e-5, out
    assert m1 < m2 and m2 > 0.98, out
