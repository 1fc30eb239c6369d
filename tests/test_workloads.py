"""The seeded generators: reproducible, chunk-independent, and with the stated structure."""
import numpy as np
import pytest

import oracle
from paper_1104_3830_gb300 import workloads as W


def test_uniform_reproducible_and_in_range():
    a = W.uniform(300, 1, 1000, 5)
    b = W.uniform(300, 1, 1000, 5)
    assert np.array_equal(a, b) and a.min() >= 1 and a.max() <= 1000
    assert not np.array_equal(a, W.uniform(300, 1, 1000, 6))
    # counter based: any element regenerates alone
    key = W.stream_key(5, 1, 0, 300)
    assert W.uniform_ints(key, 300 * 7 + 11, 1, 1, 1000)[0] == a[7, 11]
    # roughly uniform
    assert abs(a.mean() - 500.5) < 5


def test_planted_optimum_is_the_plant():
    w, pi, pairs = W.planted(64, 3)
    assert w.dtype == np.int16 and w.max() <= 10000 and w.min() >= 1
    assert np.all(w[np.arange(64), pi] == np.sort(w, axis=1)[:, -1])
    b = oracle.log_weights(w.astype(np.int64))
    assert list(oracle.hungarian(b)[0]) == list(pi)


def test_tied_pairs_disjoint():
    w, pi, pairs = W.planted(200, 4, tied_frac=0.01 * 10)
    assert pairs.shape == (10, 2) and len(set(pairs.ravel())) == 20
    for i, k in pairs:
        assert w[i, pi[k]] == w[k, pi[i]] == w[i, pi[i]] == 10000


def test_zipf_sizes_arrivals():
    z = W.zipf(64, 1.2, 30000, 1)
    assert z.min() >= 1 and z.max() <= 30000 and (z == 1).mean() > 0.2
    n = W.loguniform_sizes(4096, 16, 512, 2)
    assert n.min() >= 16 and n.max() <= 512 and abs(np.median(n) - np.sqrt(16 * 513)) < 15
    t = W.poisson_arrivals(2000.0, 2.0, 3)
    assert abs(len(t) - 4000) < 300 and np.all(np.diff(t) > 0)


def test_euclidean_generator_and_quantisation_bound():
    """The Euclidean random matrix (Sec. 5): weights in the stated range, deterministic, and
    the optimum of the quantised weights is within 2 n delta of the minimum total distance
    (delta = 0.5 / (2^20 e^-sqrt(3)), the largest error of one log weight)."""
    import math
    scipy_opt = pytest.importorskip("scipy.optimize")
    n = 60
    w, x, y = W.euclidean(n, 11)
    w2, _, _ = W.euclidean(n, 11)
    assert np.array_equal(w, w2) and w.dtype == np.int32
    assert w.min() >= int(round((1 << 20) * math.exp(-math.sqrt(3)))) and w.max() <= (1 << 20)
    d = np.sqrt(((x[:, None, :] - y[None, :, :]) ** 2).sum(axis=2))
    assert np.max(np.abs(np.log(w / float(1 << 20)) + d)) <= 0.5 / ((1 << 20) * math.exp(-math.sqrt(3)))
    r, c = scipy_opt.linear_sum_assignment(d)
    perm, _, _, st = oracle.hungarian(oracle.log_weights(w.astype(np.int64)))
    assert st == 0
    delta = 0.5 / ((1 << 20) * math.exp(-math.sqrt(3)))
    assert d[np.arange(n), perm].sum() <= d[r, c].sum() + 2 * n * delta + 1e-12
