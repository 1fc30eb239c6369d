"""Parity of the per-step FP32 matrix path (SA_KERNEL_STEP) with the FP64 oracle.

Tolerance: at the start of every p step the kernel forms each exponent
p*log2(w) - C_i - V_j in float-pair arithmetic (log2 w to about 2^-40 from a table and a
series, exact two-products and two-sums) and rounds it once to FP32 before one SFU exp2,
so every entry of the step matrix K carries a relative error of at most
2^-24 * |exponent| * ln 2 + 2^-22 (the SFU exp2 bound); the largest entries of a row have
exponents near 0.  Within the step only FP32 sums (relative error of a few 2^-24 each) and
the column factors c_j = 2^(Vs_j - V_j) (one SFU exp2 each) enter.  So, unlike the
single-read kernel whose FP32 log2 error is multiplied by p, the FP64-recomputed row and
column sums of the result stay within a bound that does not depend on p:
STEP_SUM_BOUND = 1e-6 (the stopping tol) + 1e-6 (arithmetic).
"""
import numpy as np
import pytest

import oracle
from paper_1104_3830_gb300 import api
from paper_1104_3830_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

STEP_SUM_BOUND = 2e-6


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


@pytest.mark.parametrize("n,dtype,seed", [(256, np.int32, 0), (1000, np.int16, 1), (777, np.int32, 2),
                                          (8, np.int16, 3), (1, np.int32, 4), (130, np.int16, 5),
                                          (2049, np.int16, 6), (1500, np.int16, 7), (5000, np.int16, 8)])
def test_low_p_matches_oracle_elementwise(ctx, n, dtype, seed):
    """Ragged widths (n % 4 != 0, a single row, one, two and four column chunks per
    thread: every template below the wide ones)."""
    w = W.uniform(n, 1, 1000, 900 + seed, dtype=dtype)
    ps = [1.0, 2.0, 4.0, 8.0]
    d = api.to_device(w)
    u, v, info = api.sa_scale(ctx, d, ps, 1e-6, 20000, kernel="step")
    assert info["status"] == 0 and info["kernel_used"] == 3, info
    u, v = u.cpu().numpy(), v.cpu().numpy()
    b = oracle.log_weights(w.astype(np.int64))
    uo, vo, swo, rso, sto = oracle.sinkhorn(b, ps, 1e-6, 20000)
    assert sto == 0
    xg = oracle.xmatrix(b, ps[-1], u, v)
    xo = oracle.xmatrix(b, ps[-1], uo, vo)
    # both sides stop within tol of bistochastic: entries agree to a few tol
    assert np.all(np.abs(xg - xo) <= 8e-6 * np.maximum(xo, 1.0 / max(n, 1)) + 1e-9), np.max(np.abs(xg - xo))
    assert fp64_sum_err(b, ps[-1], u, v) < STEP_SUM_BOUND


def test_c1_schedule_error_does_not_grow_with_p(ctx):
    """n = 256, int32 weights in [1, 1000], p = 1, ..., 256: the FP64-recomputed sums of the
    step path stay within a p-independent bound, and its u_i + v_j match the oracle's."""
    w, ps = W.c1()
    d = api.to_device(w)
    b = oracle.log_weights(w.astype(np.int64))
    u, v, info = api.sa_scale(ctx, d, ps, 1e-6, 20000, kernel="step")
    assert info["status"] == 0 and info["residual"] <= 1e-6, info
    u, v = u.cpu().numpy(), v.cpu().numpy()
    err = fp64_sum_err(b, ps[-1], u, v)
    assert err < STEP_SUM_BOUND, err
    er, ec = api.sa_verify(ctx, d, ps[-1], torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda())
    assert abs(max(er, ec) - err) < 1e-9
    uo, vo, swo, rso, sto = oracle.sinkhorn(b, ps, 1e-6, 20000)
    xo = oracle.xmatrix(b, ps[-1], uo, vo)
    big = xo > 1e-3
    s_g = (u[:, None] + v[None, :])[big]
    s_o = (uo[:, None] + vo[None, :])[big]
    # x = exp(p b - u - v): agreement of x within a few tol means u + v within a few tol
    assert np.max(np.abs(s_g - s_o)) < 1e-4


def test_planted_high_p_sums(ctx):
    """Planted n = 512 int16 instance up to p = 512: the step path's FP64 sums stay within
    the p-independent bound (the single-read path's would be about 1.3e-7 * p)."""
    w, pi, _ = W.planted(512, W.BASE_SEED + 40)
    ps = [2.0 ** k for k in range(10)]
    d = api.to_device(w)
    u, v, info = api.sa_scale(ctx, d, ps, 1e-6, 5000, kernel="step")
    assert info["status"] in (0, -4), info
    b = oracle.log_weights(w.astype(np.int64))
    err = fp64_sum_err(b, ps[-1], u.cpu().numpy(), v.cpu().numpy())
    assert err < max(STEP_SUM_BOUND, 2 * info["residual"] + 1e-6), (err, info["residual"])


def test_step_and_fused_agree_at_low_p(ctx):
    w = W.uniform(512, 1, 1000, 77, dtype=np.int16)
    ps = [1.0, 2.0, 4.0, 8.0]
    d = api.to_device(w)
    us, vs, _ = api.sa_scale(ctx, d, ps, 1e-6, kernel="step")
    uf, vf, _ = api.sa_scale(ctx, d, ps, 1e-6, kernel="fused")
    b = oracle.log_weights(w.astype(np.int64))
    xs = oracle.xmatrix(b, 8.0, us.cpu().numpy(), vs.cpu().numpy())
    xf = oracle.xmatrix(b, 8.0, uf.cpu().numpy(), vf.cpu().numpy())
    assert np.max(np.abs(xs - xf)) < 2e-5


def test_resume_equals_full_run(ctx):
    w = W.uniform(400, 1, 1000, 80, dtype=np.int16)
    ps = [1.0, 2.0, 4.0, 8.0, 16.0]
    d = api.to_device(w)
    u1, v1, _ = api.sa_scale(ctx, d, ps, 1e-6, kernel="step")
    u2, v2, _ = api.sa_scale(ctx, d, ps[:3], 1e-6, kernel="step")
    u3, v3, info = api.sa_scale(ctx, d, ps, 1e-6, resume_from=3, u=u2, v=v2, kernel="step")
    assert info["steps_done"] == 2 and info["kernel_used"] == 3
    b = oracle.log_weights(w.astype(np.int64))
    x1 = oracle.xmatrix(b, 16.0, u1.cpu().numpy(), v1.cpu().numpy())
    x3 = oracle.xmatrix(b, 16.0, u3.cpu().numpy(), v3.cpu().numpy())
    assert np.max(np.abs(x1 - x3)) < 2e-5


def test_auto_picks_step_for_mixed(ctx):
    w = W.uniform(300, 1, 1000, 83, dtype=np.int16)
    d = api.to_device(w)
    _, _, info = api.sa_scale(ctx, d, [1.0, 2.0], 1e-6)
    assert info["kernel_used"] == 3
    _, _, info = api.sa_scale(ctx, d, [1.0, 2.0], 1e-6, prec="fp32")
    assert info["kernel_used"] in (1, 2)


def test_zero_column_is_nonfinite(ctx):
    """A column without support is found by the column finalisation of some block; every
    block then leaves (at the next grid barrier at the latest) and the call returns
    SA_E_NONFINITE on the three-row stage ring (n = 8192) as on the smallest one."""
    for n in (256, 8192):
        w = W.uniform(n, 1, 1000, 82 + n, dtype=np.int16)
        w[:, 5] = 0
        d = api.to_device(w)
        with pytest.raises(api.SaError) as e:
            api.sa_scale(ctx, d, [1.0, 2.0], 1e-6, 50, kernel="step")
        assert e.value.status == -6, n
    w2 = W.uniform(256, 1, 1000, 85, dtype=np.int16)
    _, _, info = api.sa_scale(ctx, api.to_device(w2), [1.0, 2.0], 1e-6, kernel="step")
    assert info["status"] == 0


def test_zero_row_is_nonfinite(ctx):
    w = W.uniform(256, 1, 1000, 81, dtype=np.int16)
    w[17, :] = 0
    d = api.to_device(w)
    with pytest.raises(api.SaError) as e:
        api.sa_scale(ctx, d, [1.0, 2.0], 1e-6, 50, kernel="step")
    assert e.value.status == -6
    # the context stays usable
    w2 = W.uniform(256, 1, 1000, 84, dtype=np.int16)
    _, _, info = api.sa_scale(ctx, api.to_device(w2), [1.0, 2.0], 1e-6, kernel="step")
    assert info["status"] == 0


def max_x_deviation(b, p, u1, v1, u2, v2, rows=512):
    """max |x1 - x2| / max(x2, 1/n) over all entries, x from the definition, by row blocks."""
    n = b.shape[0]
    worst = 0.0
    for r0 in range(0, n, rows):
        bb = p * b[r0:r0 + rows]
        x1 = np.exp(bb - u1[r0:r0 + rows, None] - v1[None, :])
        x2 = np.exp(bb - u2[r0:r0 + rows, None] - v2[None, :])
        worst = max(worst, float(np.max(np.abs(x1 - x2) / np.maximum(x2, 1.0 / n))))
    return worst


def test_largest_supported_width(ctx):
    """n = 12288 (six chunks of four columns per thread, the widest ring of two-row stages:
    two stages, each consumed before the next is read): X(p) entry by entry against the
    oracle and its FP64 sums by the oracle."""
    n = 12288
    w = W.uniform(n, 1, 1000, 85, dtype=np.int16)
    d = api.to_device(w)
    ps = [1.0, 2.0]
    u, v, info = api.sa_scale(ctx, d, ps, 1e-6, 2000, kernel="step")
    assert info["status"] == 0 and info["kernel_used"] == 3, info
    u, v = u.cpu().numpy(), v.cpu().numpy()
    b = oracle.log_weights(w.astype(np.int64))
    uo, vo, _, _, st = oracle.sinkhorn(b, ps, 1e-6, 2000)
    assert st == 0
    assert max_x_deviation(b, ps[-1], u, v, uo, vo) < 8e-6
    assert fp64_sum_err(b, ps[-1], u, v) < STEP_SUM_BOUND


@pytest.mark.parametrize("n", [7001, 8500])
def test_three_row_stages(ctx, n):
    """Rows of 27 to 35 KB run through a ring of two three-row stages: a ragged width
    n = 7001 (four chunks per thread) and n = 8500 (six chunks), int16 weights in [1, 1000],
    p = 1, 2: X(p) entry by entry against the oracle and its FP64 sums by the oracle (the
    planted n = 8192 workload runs the same ring in the full-size tests)."""
    w = W.uniform(n, 1, 1000, 88 + n, dtype=np.int16)
    d = api.to_device(w)
    ps = [1.0, 2.0]
    u, v, info = api.sa_scale(ctx, d, ps, 1e-6, 2000, kernel="step")
    assert info["status"] == 0 and info["kernel_used"] == 3, info
    uu, vv = u.cpu().numpy(), v.cpu().numpy()
    b = oracle.log_weights(w.astype(np.int64))
    uo, vo, _, _, st = oracle.sinkhorn(b, ps, 1e-6, 2000)
    assert st == 0
    assert max_x_deviation(b, ps[-1], uu, vv, uo, vo, rows=512) < 8e-6
    assert fp64_sum_err(b, ps[-1], uu, vv) < STEP_SUM_BOUND


@pytest.mark.parametrize("n", [12290, 22000])
def test_wide_rows_one_row_stages(ctx, n):
    """Rows of more than 48 KB run through a ring of one-row stages: a ragged width
    n = 12290 (eight chunks per thread, three slots, partial row sums formed one stage
    ahead) and n = 22000 (twelve chunks, the widest; two slots, each stage consumed before
    the next is read), int16 weights in [1, 32767], p = 1, 2, 4: X(p) entry by entry against
    the oracle and its FP64 sums by the oracle (n = 20000, ten chunks, runs in the
    full-size tests)."""
    w = W.uniform(n, 1, 32767, 86, dtype=np.int16)
    d = api.to_device(w)
    ps = [1.0, 2.0, 4.0]
    u, v, info = api.sa_scale(ctx, d, ps, 1e-6, 2000, kernel="step")
    assert info["status"] == 0 and info["kernel_used"] == 3, info
    uu, vv = u.cpu().numpy(), v.cpu().numpy()
    b = oracle.log_weights(w.astype(np.int64))
    uo, vo, _, _, st = oracle.sinkhorn(b, ps, 1e-6, 2000)
    assert st == 0
    assert max_x_deviation(b, ps[-1], uu, vv, uo, vo, rows=256) < 8e-6
    assert fp64_sum_err(b, ps[-1], uu, vv) < STEP_SUM_BOUND
    with pytest.raises(api.SaError):
        api.sa_scale(ctx, api.to_device(W.uniform(24580, 1, 10, 87, dtype=np.int16)), [1.0], 1e-6, 10,
                     kernel="step")


def _ctx_with(**options):
    c = api.sa_create(0)
    for name, value in options.items():
        api.sa_set_option(c, name, value)
    return c


@pytest.mark.parametrize("n", [512, 2048])
def test_sparse_epochs_match_dense(ctx, n):
    """At high p most entries of the step matrix fall below 2^-70 of their row and the step
    path sweeps only the rest.  Same potentials (as X) as the all-dense path within a few
    tol, FP64 sums within the p-independent bound."""
    w, pi, _ = W.planted(n, W.BASE_SEED + 41 + n)
    ps = [2.0 ** k for k in range(10)]
    d = api.to_device(w)
    sp = _ctx_with(step_sparse=1)
    dense = _ctx_with(step_sparse=0)
    try:
        us, vs, info_s = api.sa_scale(sp, d, ps, 1e-6, 3000, kernel="step")
        ud, vd, info_d = api.sa_scale(dense, d, ps, 1e-6, 3000, kernel="step")
    finally:
        sp.close()
        dense.close()
    assert info_s["sparse_epochs"] > 0, info_s
    assert info_d["sparse_epochs"] == 0, info_d
    b = oracle.log_weights(w.astype(np.int64))
    us, vs, ud, vd = us.cpu().numpy(), vs.cpu().numpy(), ud.cpu().numpy(), vd.cpu().numpy()
    for (u, v, info) in ((us, vs, info_s), (ud, vd, info_d)):
        err = fp64_sum_err(b, ps[-1], u, v)
        assert err < max(STEP_SUM_BOUND, 2 * info["residual"] + 1e-6), (err, info)
    xs = oracle.xmatrix(b, ps[-1], us, vs)
    xd = oracle.xmatrix(b, ps[-1], ud, vd)
    tol_x = 4 * max(info_s["residual"], info_d["residual"], 1e-6) + 1e-6
    assert np.max(np.abs(xs - xd)) < tol_x, np.max(np.abs(xs - xd))
    # the planted permutation carries the mass at p = 512
    assert np.all(xs[np.arange(n), pi] > 0.5)
