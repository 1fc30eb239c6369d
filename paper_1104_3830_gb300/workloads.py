"""Seeded synthetic inputs for the assignment workloads.

This module holds only random-number generation and input layout: none of the
method's arithmetic.  Both the CUDA path's tests and the FP64 oracle draw from it, so
the two sides always see bit-identical matrices.

Randomness is counter based: every draw is SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) of a stream key plus a
counter, so any element can be regenerated alone and the result does not depend on
how the work is chunked.

Workloads (n x n integer weights w_ij >= 1, a_ij = w_ij):

* ``uniform(n, lo, hi, seed)``      i.i.d. uniform integers in [lo, hi]
* ``planted(n, seed, tied_frac)``   uniform off-plan weights in [1, 9500]; a hidden
                                    permutation pi gets, in each row, that row's largest
                                    off-plan weight + 500, so pi is the unique optimum;
                                    with tied_frac > 0, floor(tied_frac*n/2) disjoint row
                                    pairs get all four cross entries at 10000, making
                                    2^pairs optimal permutations
* ``zipf(n, s, hi, seed)``          Zipf(s) weights on {1..hi} by inverse CDF
* ``euclidean(n, seed)``            the Euclidean random matrix of the paper's experiments:
                                    2n points uniform in the unit cube, a_ij =
                                    exp(-|x_i - y_j|), quantised to integers
                                    w_ij = round(2^20 a_ij) (in [185000, 2^20])
* ``loguniform_sizes(k, lo, hi, seed)`` instance sizes floor(exp(U(ln lo, ln(hi+1))))
* ``poisson_arrivals(rate, duration, seed)`` arrival times with exponential gaps
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on uint64 arrays (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def stream_key(seed: int, *tags: int) -> np.uint64:
    """Derive an independent stream key from a seed and integer tags."""
    k = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    for t in tags:
        with np.errstate(over="ignore"):
            k = _mix(np.array([k ^ np.uint64(t & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64)
                     + _GOLDEN)[0]
    return k


def bits(key: np.uint64, start: int, count: int) -> np.ndarray:
    """count 64-bit draws with counters start..start+count-1 of stream key."""
    ctr = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + (ctr + np.uint64(1)) * _GOLDEN)


def uniform_ints(key, start, count, lo, hi) -> np.ndarray:
    """Integers in [lo, hi] from the top 32 bits (multiply-shift range reduction)."""
    span = np.uint64(hi - lo + 1)
    r = (bits(key, start, count) >> np.uint64(32)) * span >> np.uint64(32)
    return (r.astype(np.int64) + lo)


def uniform01(key, start, count) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits."""
    return (bits(key, start, count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def uniform(n: int, lo: int, hi: int, seed: int, dtype=np.int32, tag: int = 0) -> np.ndarray:
    """n x n weights uniform in [lo, hi], row-major."""
    key = stream_key(seed, 1, tag, n)
    out = np.empty((n, n), dtype=dtype)
    rows_per = max(1, (1 << 24) // max(n, 1))
    for r0 in range(0, n, rows_per):
        r1 = min(n, r0 + rows_per)
        out[r0:r1] = uniform_ints(key, r0 * n, (r1 - r0) * n, lo, hi).reshape(r1 - r0, n)
    return out


def permutation(n: int, key) -> np.ndarray:
    """A uniformly random permutation: argsort of n independent 64-bit keys."""
    return np.argsort(bits(key, 0, n), kind="stable").astype(np.int64)


def planted(n: int, seed: int, tied_frac: float = 0.0, dtype=np.int16):
    """Weights with a planted optimal permutation pi (returned with the matrix).

    Off-plan entries are uniform in [1, 9500]; w[i, pi[i]] = max_{j != pi[i]} w[i, j] + 500
    <= 10000, the strict maximum of its row, so pi is the unique optimum.  With
    tied_frac > 0, floor(tied_frac * n / 2) disjoint pairs of rows (i, k) get
    w[i, pi[i]] = w[i, pi[k]] = w[k, pi[i]] = w[k, pi[k]] = 10000.
    Returns (w, pi, pairs) with pairs an (m, 2) array of the tied row pairs."""
    w = uniform(n, 1, 9500, seed, dtype=np.int32, tag=2)
    pi = permutation(n, stream_key(seed, 3, n))
    rows = np.arange(n)
    w[rows, pi] = 0
    w[rows, pi] = w.max(axis=1) + 500
    m = int(np.floor(tied_frac * n / 2))
    pairs = np.zeros((0, 2), dtype=np.int64)
    if m > 0:
        order = permutation(n, stream_key(seed, 4, n))
        pairs = order[: 2 * m].reshape(m, 2)
        for i, k in pairs:
            for r in (i, k):
                for c in (pi[i], pi[k]):
                    w[r, c] = 10000
    return w.astype(dtype), pi, pairs


def zipf(n: int, s: float, hi: int, seed: int, dtype=np.int16, tag: int = 0) -> np.ndarray:
    """n x n weights with P(w = k) proportional to k^-s on {1..hi} (inverse CDF)."""
    k = np.arange(1, hi + 1, dtype=np.float64)
    cdf = np.cumsum(k ** (-s))
    cdf /= cdf[-1]
    key = stream_key(seed, 5, tag, n)
    u = uniform01(key, 0, n * n)
    idx = np.searchsorted(cdf, u, side="right")
    return (np.minimum(idx, hi - 1) + 1).astype(dtype).reshape(n, n)


def euclidean(n: int, seed: int, scale: int = 1 << 20):
    """n x n int32 weights round(scale * exp(-|x_i - y_j|)) for points x_i, y_j uniform in
    the unit cube of R^3 (the Euclidean random matrix of the paper's experiments), and the
    points (x, y).  The weights are the input's definition, quantised so that the integer
    kernels take them: an optimum of w is within n * 1.1e-5 of the optimal total distance
    (each log w is within 0.5 / (scale * e^-sqrt(3)) of -d)."""
    key = stream_key(seed, 6, n)
    pts = uniform01(key, 0, 6 * n).reshape(2, n, 3)
    x, y = pts[0], pts[1]
    d = np.sqrt(((x[:, None, :] - y[None, :, :]) ** 2).sum(axis=2))
    w = np.maximum(1, np.rint(scale * np.exp(-d))).astype(np.int32)
    return w, x, y


def loguniform_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Sizes floor(exp(U(ln lo, ln(hi + 1)))) clipped to [lo, hi]."""
    u = uniform01(stream_key(seed, 6, count), 0, count)
    n = np.floor(np.exp(np.log(lo) + u * (np.log(hi + 1) - np.log(lo)))).astype(np.int64)
    return np.clip(n, lo, hi)


def poisson_arrivals(rate: float, duration: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate on [0, duration)."""
    expected = int(rate * duration * 1.2 + 100)
    u = uniform01(stream_key(seed, 7), 0, expected)
    gaps = -np.log1p(-u) / rate
    t = np.cumsum(gaps)
    return t[t < duration]


# The five workload shapes, seed = 20261202 + index.
BASE_SEED = 20261202


def c1(seed: int = BASE_SEED + 0):
    """n = 256, int32 weights uniform in [1, 1000], p in {1, 2, ..., 256}."""
    return uniform(256, 1, 1000, seed, dtype=np.int32), [2.0 ** k for k in range(9)]


def c2(seed: int = BASE_SEED + 1, n: int = 8192, tied_frac: float = 0.0):
    """n = 8192 int16 planted, p in {1, ..., 512}."""
    w, pi, pairs = planted(n, seed, tied_frac)
    return w, [2.0 ** k for k in range(10)], pi, pairs


def c3(seed: int = BASE_SEED + 2, n: int = 20000):
    """n = 20000 int16 uniform in [1, 32767], p in {1, ..., 256}."""
    return uniform(n, 1, 32767, seed, dtype=np.int16), [2.0 ** k for k in range(9)]


def c4(seed: int = BASE_SEED + 3, count: int = 4096, lo: int = 16, hi: int = 512):
    """count instances, n log-uniform in [lo, hi], int32 uniform [1, 1000], p in {1..128}."""
    sizes = loguniform_sizes(count, lo, hi, seed)
    mats = [uniform(int(n), 1, 1000, seed, dtype=np.int32, tag=1000 + k)
            for k, n in enumerate(sizes)]
    return mats, [2.0 ** k for k in range(8)]


def c5_request(seed: int, k: int, n: int, dist: str = "uniform"):
    """The k-th request of the serving stream: uniform [1, 1000] or Zipf(1.2) on [1, 30000]."""
    if dist == "uniform":
        return uniform(n, 1, 1000, seed, dtype=np.int16, tag=5000 + k)
    return zipf(n, 1.2, 30000, seed, dtype=np.int16, tag=5000 + k)
