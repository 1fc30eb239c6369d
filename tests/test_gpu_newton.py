"""Parity of the Newton scaling path (SA_KERNEL_NEWTON, Sec. 5.3) with the FP64 oracle.

Both sides converge to X(p), the unique bistochastic matrix diagonally equivalent to
A^(p) (Sec. 2.1), by different iterations: the oracle by exact Newton steps on A^(p), the
GPU by inexact (conjugate-gradient) Newton steps on the per-step FP32 matrix K.  So X(p)
is compared entry by entry.  The GPU stops when max(|row sum - 1|, |column sum - 1|) <= tol
for sums of FP32 products of K in FP64; each entry of K carries a relative error of about
2^-24 (one rounding of an FP64 exponent) plus the FP32 exp2 bound (2 ulp), so the
FP64-recomputed sums of the result are within tol + 1e-6 (NEWTON_SUM_BOUND), and two
matrices that are bistochastic to that accuracy agree entry-wise to a few times it
(relative to max(x, 1/n)) when the instance is well conditioned, as these are.
"""
import numpy as np
import pytest

import oracle
from paper_1104_3830_gb300 import api
from paper_1104_3830_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NEWTON_SUM_BOUND = 2e-6


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_3830_gb300 import build
    build.build()
    c = api.sa_create(0)
    yield c
    c.close()


def fp64_sum_err(b, p, u, v):
    r, c = oracle.sums(b, p, u, v)
    return max(np.abs(r - 1).max(), np.abs(c - 1).max())


def close(xg, xo, n, rel=8e-6):
    return np.all(np.abs(xg - xo) <= rel * np.maximum(xo, 1.0 / max(n, 1)) + 1e-9)


@pytest.mark.parametrize("n,dtype,p,seed", [(64, np.int32, 1.0, 0), (64, np.int32, 10.0, 1), (130, np.int16, 5.0, 2),
                                            (9, np.int16, 2.0, 3), (1, np.int32, 3.0, 4), (150, np.int32, 40.0, 5)])
def test_single_p_matches_newton_oracle(ctx, n, dtype, p, seed):
    w = W.uniform(n, 1, 1000, 1500 + seed, dtype=dtype)
    d = api.to_device(w)
    u, v, info = api.sa_scale(ctx, d, [p], 1e-6, 500, kernel="newton")
    assert info["status"] == 0 and info["kernel_used"] == 4, info
    assert info["residual"] <= 1e-6
    b = oracle.log_weights(w.astype(np.int64))
    uo, vo, it, res, st = oracle.newton(b, p)
    assert st == 0
    xg = oracle.xmatrix(b, p, u.cpu().numpy(), v.cpu().numpy())
    xo = oracle.xmatrix(b, p, uo, vo)
    assert close(xg, xo, n), np.max(np.abs(xg - xo))
    assert fp64_sum_err(b, p, u.cpu().numpy(), v.cpu().numpy()) < NEWTON_SUM_BOUND


@pytest.mark.parametrize("n,dtype,seed", [(1000, np.int16, 10), (777, np.int32, 11), (2049, np.int16, 12),
                                          (4500, np.int16, 13), (5001, np.int32, 14)])
def test_schedule_matches_sinkhorn_oracle(ctx, n, dtype, seed):
    """Ragged widths, one to three float4 chunks per thread, one and two column tiles."""
    w = W.uniform(n, 1, 1000, 1600 + seed, dtype=dtype)
    ps = [1.0, 2.0, 4.0, 8.0]
    d = api.to_device(w)
    u, v, info = api.sa_scale(ctx, d, ps, 1e-6, 500, kernel="newton")
    assert info["status"] == 0 and info["kernel_used"] == 4, info
    u, v = u.cpu().numpy(), v.cpu().numpy()
    b = oracle.log_weights(w.astype(np.int64))
    uo, vo, sw, rs, st = oracle.sinkhorn(b, ps, 1e-9, 20000)
    assert st == 0
    xg = oracle.xmatrix(b, ps[-1], u, v)
    xo = oracle.xmatrix(b, ps[-1], uo, vo)
    assert close(xg, xo, n), np.max(np.abs(xg - xo))
    assert fp64_sum_err(b, ps[-1], u, v) < NEWTON_SUM_BOUND


def test_c1_schedule_to_p256(ctx):
    """n = 256, int32 weights in [1, 1000], p = 1, ..., 256 (the warm-started schedule up to
    p (b_max - b_min) = 1768, beyond the range of an explicit A^(p) in FP64)."""
    w, ps = W.c1()
    d = api.to_device(w)
    b = oracle.log_weights(w.astype(np.int64))
    u, v, info = api.sa_scale(ctx, d, ps, 1e-6, 2000, kernel="newton")
    assert info["status"] == 0 and info["residual"] <= 1e-6, info
    u, v = u.cpu().numpy(), v.cpu().numpy()
    assert fp64_sum_err(b, ps[-1], u, v) < NEWTON_SUM_BOUND
    uo, vo, _, _, sto = oracle.sinkhorn(b, ps, 1e-9, 200000)
    assert sto == 0
    xg = oracle.xmatrix(b, ps[-1], u, v)
    xo = oracle.xmatrix(b, ps[-1], uo, vo)
    assert np.max(np.abs(xg - xo)) < 2e-4, np.max(np.abs(xg - xo))


def test_planted_high_p_fewer_operator_reads_than_sinkhorn(ctx):
    """Planted instance (unique optimum, Sec. 3.1): as p grows X(p) approaches the
    permutation matrix and Sinkhorn slows down (its rate is the second singular value of
    X); the Newton path converges in far fewer reads of K.  Both end at the same X."""
    w, perm, _ = W.planted(1024, 77, dtype=np.int16)
    ps = [2.0 ** k for k in range(0, 9)]
    d = api.to_device(w)
    un, vn, infn = api.sa_scale(ctx, d, ps, 1e-6, 20000, kernel="newton")
    us, vs, infs = api.sa_scale(ctx, d, ps, 1e-6, 20000, kernel="step")
    assert infn["status"] == 0, infn
    assert infs["status"] in (0, -4), infs   # Sinkhorn may reach its cap at the top p
    print("newton matvecs", infn["sweeps_total"], "step sweeps", infs["sweeps_total"])
    assert infn["sweeps_total"] < infs["sweeps_total"]
    er, ec = api.sa_verify(ctx, d, ps[-1], un, vn)
    assert max(er, ec) < NEWTON_SUM_BOUND
    b = oracle.log_weights(w.astype(np.int64))
    xn = oracle.xmatrix(b, ps[-1], un.cpu().numpy(), vn.cpu().numpy())
    xs = oracle.xmatrix(b, ps[-1], us.cpu().numpy(), vs.cpu().numpy())
    if infs["status"] == 0:
        assert np.max(np.abs(xn - xs)) < 1e-4
    assert np.all(np.argmax(xn, axis=1) == perm)


def test_resume_equals_full_run(ctx):
    w = W.uniform(400, 1, 1000, 1680, dtype=np.int16)
    ps = [1.0, 2.0, 4.0, 8.0, 16.0]
    d = api.to_device(w)
    u1, v1, _ = api.sa_scale(ctx, d, ps, 1e-6, kernel="newton")
    u2, v2, _ = api.sa_scale(ctx, d, ps[:3], 1e-6, kernel="newton")
    u3, v3, info = api.sa_scale(ctx, d, ps, 1e-6, resume_from=3, u=u2, v=v2, kernel="newton")
    assert info["steps_done"] == 2 and info["kernel_used"] == 4
    b = oracle.log_weights(w.astype(np.int64))
    x1 = oracle.xmatrix(b, 16.0, u1.cpu().numpy(), v1.cpu().numpy())
    x3 = oracle.xmatrix(b, 16.0, u3.cpu().numpy(), v3.cpu().numpy())
    assert np.max(np.abs(x1 - x3)) < 2e-5


def test_cap_reports_not_converged(ctx):
    w = W.uniform(300, 1, 1000, 1681, dtype=np.int16)
    d = api.to_device(w)
    _, _, info = api.sa_scale(ctx, d, [30.0], 1e-9, 3, kernel="newton")
    assert info["status"] == -4 and info["converged"] == 0
    assert info["sweeps_total"] <= 4


def test_zero_column_is_nonfinite(ctx):
    w = W.uniform(256, 1, 1000, 1682, dtype=np.int16)
    w[:, 40] = 0
    d = api.to_device(w)
    with pytest.raises(api.SaError) as e:
        api.sa_scale(ctx, d, [1.0, 2.0], 1e-6, 50, kernel="newton")
    assert e.value.status == -6
    w2 = W.uniform(256, 1, 1000, 1683, dtype=np.int16)
    _, _, info = api.sa_scale(ctx, api.to_device(w2), [1.0, 2.0], 1e-6, kernel="newton")
    assert info["status"] == 0


def test_newton_needs_mixed_precision(ctx):
    w = W.uniform(64, 1, 1000, 1684, dtype=np.int16)
    with pytest.raises(api.SaError):
        api.sa_scale(ctx, api.to_device(w), [1.0], 1e-6, kernel="newton", prec="fp32")


@pytest.mark.parametrize("n", [12290, 20000, 24576])
def test_wide_matrices_fp64_sums(ctx, n):
    """Four to six column tiles (n = 12290 ragged): FP64 row and column sums of the result
    by the library's own verification, the property that holds at any size."""
    w = W.uniform(n, 1, 1000, 1690 + n % 97, dtype=np.int16)
    d = api.to_device(w)
    u, v, info = api.sa_scale(ctx, d, [1.0, 2.0], 1e-6, 500, kernel="newton")
    assert info["status"] == 0 and info["kernel_used"] == 4, info
    er, ec = api.sa_verify(ctx, d, 2.0, u, v)
    assert max(er, ec) < NEWTON_SUM_BOUND, (er, ec)
    # sampled rows against the definition x_ij = exp(p b_ij - u_i - v_j) in FP64
    uu, vv = u.cpu().numpy(), v.cpu().numpy()
    for i in (0, n // 3, n - 1):
        row = np.exp(2.0 * np.log(w[i].astype(np.float64)) - uu[i] - vv)
        assert abs(row.sum() - 1.0) < NEWTON_SUM_BOUND
