"""Parity of the default scaling path with the FP64 oracle at the benchmark's own sizes.

The step kernel has one template per width class (chunks of four columns per thread);
the sizes here are the ones the benchmark runs, so each template the planted n = 8192
workload and the n = 20000 precision workload use is compared with the oracle itself,
not with the library's own FP64 check:

* n = 8192 (four chunks per thread, rows through the shared-memory ring): X(p) entry by
  entry against ``oracle.sinkhorn`` over p = 1 ... 32 (the oracle needs two or three
  sweeps per step there), then the whole p = 1 ... 512 schedule of the benchmark, where
  the oracle cannot follow the 20000 sweeps of the p = 256 step: FP64 row and column sums
  of the result by ``oracle.sums`` (Sec. 4.2: the result is eps-bistochastic), the
  planted permutation carrying the mass (X(p) tends to the optimal permutation matrix,
  Sec. 3.1), and the exact optimum of ``sa_assign`` against the planted optimum.
* n = 20000 (ten chunks per thread, rows of 80 KB through a ring of two one-row stages):
  X(p) entry by entry against ``oracle.sinkhorn`` at p = 1, 2 and the FP64 sums by
  ``oracle.sums``.

Tolerances: as in the other step-kernel tests, entries within 8e-6 max(x, 1/n) of the
oracle's (both sides stop within tol = 1e-6 of bistochastic, measured on different sums)
and FP64 sums within 2e-6, or within twice the reported residual plus 1e-6 for a step
that stopped at its sweep cap.
"""
import numpy as np
import pytest

import oracle
from paper_1104_3830_gb300 import api
from paper_1104_3830_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEP_SUM_BOUND = 2e-6
X_REL = 8e-6


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_3830_gb300 import build
    build.build()
    c = api.sa_create(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def c2():
    w, ps, pi, _ = W.c2()
    return w, ps, pi, oracle.log_weights(w.astype(np.int64))


def max_x_deviation(b, p, u1, v1, u2, v2, rows=512):
    """max over all entries of |x1 - x2| / max(x2, 1/n), x = exp(p b - u - v) from the
    definition, in blocks of rows (the full matrix of a wide instance is gigabytes)."""
    n = b.shape[0]
    worst = 0.0
    for r0 in range(0, n, rows):
        bb = p * b[r0:r0 + rows]
        x1 = np.exp(bb - u1[r0:r0 + rows, None] - v1[None, :])
        x2 = np.exp(bb - u2[r0:r0 + rows, None] - v2[None, :])
        worst = max(worst, float(np.max(np.abs(x1 - x2) / np.maximum(x2, 1.0 / n))))
    return worst


def fp64_sum_err(b, p, u, v):
    r, c = oracle.sums(b, p, u, v)
    return max(float(np.abs(r - 1).max()), float(np.abs(c - 1).max()))


def test_c2_matches_oracle_elementwise(ctx, c2):
    w, _, _, b = c2
    ps = [1.0, 2.0, 4.0, 8.0, 16.0, 32.0]
    u, v, info = api.sa_scale(ctx, api.to_device(w), ps, 1e-6, 20000, kernel="step")
    assert info["status"] == 0 and info["kernel_used"] == 3, info
    u, v = u.cpu().numpy(), v.cpu().numpy()
    uo, vo, _, _, st = oracle.sinkhorn(b, ps, 1e-6, 20000)
    assert st == 0
    dev = max_x_deviation(b, ps[-1], u, v, uo, vo)
    assert dev < X_REL, dev
    assert fp64_sum_err(b, ps[-1], u, v) < STEP_SUM_BOUND


def test_c2_benchmark_schedule(ctx, c2):
    """p = 1, 2, ..., 512 with tol 1e-6 and the 20000-sweep cap, as the benchmark runs it."""
    w, ps, pi, b = c2
    n = w.shape[0]
    d = api.to_device(w)
    u, v, info = api.sa_scale(ctx, d, ps, 1e-6, 20000, kernel="step")
    assert info["status"] in (0, -4) and info["kernel_used"] == 3, info
    u, v = u.cpu().numpy(), v.cpu().numpy()
    err = fp64_sum_err(b, ps[-1], u, v)
    assert err < max(STEP_SUM_BOUND, 2 * info["residual"] + 1e-6), (err, info["residual"])
    rows = np.arange(n)
    x_plan = np.exp(ps[-1] * b[rows, pi] - u - v[pi])
    assert np.all(x_plan > 0.5), float(x_plan.min())
    res = api.sa_assign(ctx, d, ps, 1e-6, 20000)
    assert np.array_equal(res["perm"], pi)
    assert oracle.perm_weight_exact(w, res["perm"]) == oracle.perm_weight_exact(w, pi)


def test_c2_tied_variant(ctx):
    """The 1 % tied variant: 2^pairs optimal permutations, all of the planted weight."""
    w, ps, pi, pairs = W.c2(tied_frac=0.01)
    assert len(pairs) > 0
    b = oracle.log_weights(w.astype(np.int64))
    d = api.to_device(w)
    u, v, info = api.sa_scale(ctx, d, ps, 1e-6, 2000, kernel="step")
    assert info["status"] in (0, -4), info
    err = fp64_sum_err(b, ps[-1], u.cpu().numpy(), v.cpu().numpy())
    assert err < max(STEP_SUM_BOUND, 2 * info["residual"] + 1e-6), (err, info["residual"])
    res = api.sa_assign(ctx, d, ps, 1e-6, 2000)
    assert sorted(res["perm"]) == list(range(w.shape[0]))
    assert oracle.perm_weight_exact(w, res["perm"]) == oracle.perm_weight_exact(w, pi)


def test_c3_wide_rows_match_oracle(ctx):
    """n = 20000, int16 weights uniform in [1, 32767] (the precision workload's matrix)."""
    w, _ = W.c3()
    b = oracle.log_weights(w.astype(np.int64))
    ps = [1.0, 2.0]
    u, v, info = api.sa_scale(ctx, api.to_device(w), ps, 1e-6, 2000, kernel="step")
    assert info["status"] == 0 and info["kernel_used"] == 3, info
    u, v = u.cpu().numpy(), v.cpu().numpy()
    uo, vo, _, _, st = oracle.sinkhorn(b, ps, 1e-6, 2000)
    assert st == 0
    dev = max_x_deviation(b, ps[-1], u, v, uo, vo, rows=256)
    assert dev < X_REL, dev
    assert fp64_sum_err(b, ps[-1], u, v) < STEP_SUM_BOUND
