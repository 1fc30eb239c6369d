"""Pins of the oracle's Newton scaling (Sec. 5.3) to facts that do not come from it.

The limit of any correct scaling method is X(p), the unique bistochastic matrix
diagonally equivalent to A^(p) (Sec. 2.1), so the Newton oracle is pinned to the
printed 3x3 X(10), to the 2x2 closed form, to rank-one inputs and to the separately
pinned Sinkhorn oracle; the quadratic rate pins its Jacobian (a dropped or mis-signed
term of the Newton equation still converges at best linearly).
"""
import math

import numpy as np
import pytest

import oracle


def _x(b, p, **kw):
    u, v, it, res, st = oracle.newton(b, p, **kw)
    assert st == 0, res
    return oracle.xmatrix(b, p, u, v), it, res


def test_newton_3x3_matches_printed_x10(golden):
    g = golden("example_3x3.txt")
    a = np.array(g["A"])
    a[1, 2] = 1.0 / 3.0
    x, _, _ = _x(oracle.log_weights(a), g["p"])
    assert np.max(np.abs(x - np.array(g["X"]))) < 1e-4


@pytest.mark.parametrize("seed", range(4))
def test_newton_2x2_closed_form(seed):
    rng = np.random.default_rng(100 + seed)
    a = rng.uniform(0.1, 3.0, size=(2, 2))
    b = oracle.log_weights(a)
    for p in (0.5, 2.0, 9.0):
        x, _, _ = _x(b, p)
        k = (a[0, 0] * a[1, 1] / (a[0, 1] * a[1, 0])) ** p
        s = math.sqrt(k) / (1 + math.sqrt(k))
        assert np.allclose(x, [[s, 1 - s], [1 - s, s]], atol=1e-12, rtol=0)


def test_newton_rank_one_is_uniform():
    rng = np.random.default_rng(7)
    r, c = rng.uniform(0.5, 5, 6), rng.uniform(0.5, 5, 6)
    b = oracle.log_weights(np.outer(r, c))
    for p in (1.0, 20.0):
        x, _, _ = _x(b, p)
        assert np.allclose(x, 1 / 6, atol=1e-12)


@pytest.mark.parametrize("p", [1.0, 4.0, 25.0])
def test_newton_equals_sinkhorn_limit(p):
    rng = np.random.default_rng(11)
    a = rng.uniform(1, 1000, size=(30, 30))
    a[rng.uniform(size=a.shape) < 0.2] = 0.0   # forbidden entries; the diagonal keeps support
    np.fill_diagonal(a, rng.uniform(1, 1000, 30))
    b = oracle.log_weights(a)
    x, _, _ = _x(b, p)
    us, vs, _, _, st = oracle.sinkhorn(b, [p], 1e-13, 400000)
    assert st == 0
    xs = oracle.xmatrix(b, p, us, vs)
    assert np.max(np.abs(x - xs)) < 1e-10
    assert np.all(x[a == 0] == 0)


def test_newton_rate_is_quadratic():
    rng = np.random.default_rng(12)
    b = oracle.log_weights(rng.uniform(1, 1000, size=(40, 40)))
    for p in (1.0, 10.0, 30.0):
        _, it, res = _x(b, p)
        pairs = [(res[k], res[k + 1]) for k in range(len(res) - 1) if res[k] < 0.1 and res[k + 1] > 1e-13]
        assert pairs, res
        for r0, r1 in pairs:
            assert r1 <= 2.0 * r0 * r0, res
        assert it <= 10


def test_newton_diagonal_invariance_and_transpose():
    rng = np.random.default_rng(13)
    a = rng.uniform(1, 100, size=(8, 8))
    d1, d2 = rng.uniform(0.1, 10, 8), rng.uniform(0.1, 10, 8)
    p = 3.0
    x, _, _ = _x(oracle.log_weights(a), p)
    # X(D1 A^(p) D2) = X(A^(p)): in log form b + (log d1_i + log d2_j) / p
    bd = oracle.log_weights(a) + (np.log(d1)[:, None] + np.log(d2)[None, :]) / p
    xd, _, _ = _x(bd, p)
    assert np.allclose(x, xd, atol=1e-11)
    xt, _, _ = _x(oracle.log_weights(a.T), p)
    assert np.allclose(xt, x.T, atol=1e-11)


def test_newton_range_limit_of_explicit_powers():
    b = oracle.log_weights(np.array([[1.0, 1000.0], [2.0, 3.0]]))
    with pytest.raises(ValueError):
        oracle.newton(b, 200.0)   # p ln(1000) = 1381 > 700 (Sec. 4.1.1)
