"""Parity of the CUDA scaling path (sa_scale through the C ABI) with the FP64 oracle.

Tolerances follow from the arithmetic of the MIXED path: each exponent p*log2(w) is
formed from the SFU's FP32 log2, whose absolute error is below 1.0e-6 for every int16
input (9.8e-7 measured on GB300 over all of 1..32767), so the kernel scales a matrix whose
entries carry a relative perturbation of at most p*ln2*1.0e-6; both sides stop at the
residual tol.  X(p) is compared elementwise at moderate p and through FP64-recomputed
row and column sums at every p.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1104_3830_gb300 import api
from paper_1104_3830_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def lg_err_bound(p):
    """Relative perturbation of x_ij(p) from the FP32 exponent (see module doc)."""
    return p * math.log(2) * 1.0e-6


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_3830_gb300 import build
    build.build()
    c = api.sa_create(0)
    yield c
    c.close()


def run_both(ctx, w, ps, tol=1e-6, prec="mixed", kernel="auto", sweeps=20000):
    d = api.to_device(w)
    u, v, info = api.sa_scale(ctx, d, ps, tol, sweeps, prec=prec, kernel=kernel)
    b = oracle.log_weights(w.astype(np.int64))
    uo, vo, swo, rso, sto = oracle.sinkhorn(b, ps, tol, sweeps)
    return d, u.cpu().numpy(), v.cpu().numpy(), info, b, uo, vo, swo, sto


@pytest.mark.parametrize("kernel", ["fused", "plain"])
@pytest.mark.parametrize("n,dtype,seed", [(256, np.int32, 0), (1000, np.int16, 1), (777, np.int32, 2),
                                          (8, np.int16, 3), (1, np.int32, 4), (130, np.int16, 5)])
def test_low_p_matches_oracle_elementwise(ctx, kernel, n, dtype, seed):
    w = W.uniform(n, 1, 1000, 900 + seed, dtype=dtype)
    ps = [1.0, 2.0, 4.0, 8.0]
    d, u, v, info, b, uo, vo, swo, sto = run_both(ctx, w, ps, tol=1e-6, kernel=kernel)
    assert info["status"] == 0 and sto == 0, info
    assert info["kernel_used"] == (1 if kernel == "fused" else 2)
    xg = oracle.xmatrix(b, ps[-1], u, v)
    xo = oracle.xmatrix(b, ps[-1], uo, vo)
    bound = 4 * lg_err_bound(ps[-1]) + 4e-6
    assert np.all(np.abs(xg - xo) <= bound * xo + 5e-6), np.max(np.abs(xg - xo))
    r, c = oracle.sums(b, ps[-1], u, v)
    assert max(np.abs(r - 1).max(), np.abs(c - 1).max()) < bound


@pytest.mark.parametrize("kernel", ["fused", "plain"])
def test_c1_schedule_to_256(ctx, kernel):
    """The n = 256 instance, int32 weights in [1, 1000], p = 1, 2, ..., 256, tol 1e-6."""
    w, ps = W.c1()
    d, u, v, info, b, uo, vo, swo, sto = run_both(ctx, w, ps, kernel=kernel)
    assert info["status"] == 0, info
    assert info["residual"] <= 1e-6
    # FP64-recomputed sums of the GPU potentials: within the FP32-exponent bound
    r, c = oracle.sums(b, ps[-1], u, v)
    err = max(np.abs(r - 1).max(), np.abs(c - 1).max())
    assert err < 2 * lg_err_bound(ps[-1]) + 2e-6, err
    # the library's own FP64 verification agrees with the oracle's
    er, ec = api.sa_verify(ctx, d, ps[-1], torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda())
    assert abs(max(er, ec) - err) < 1e-9
    # gauge-invariant potentials u_i + v_j on the entries that carry mass
    xo = oracle.xmatrix(b, ps[-1], uo, vo)
    big = xo > 1e-3
    s_g = (u[:, None] + v[None, :])[big]
    s_o = (uo[:, None] + vo[None, :])[big]
    assert np.max(np.abs(s_g - s_o)) < 50 * lg_err_bound(ps[-1]) + 1e-4


def test_fused_and_plain_agree(ctx):
    w = W.uniform(512, 1, 1000, 77, dtype=np.int16)
    ps = [1.0, 2.0, 4.0, 8.0, 16.0, 32.0]
    d = api.to_device(w)
    uf, vf, inf_f = api.sa_scale(ctx, d, ps, 1e-6, kernel="fused")
    up, vp, inf_p = api.sa_scale(ctx, d, ps, 1e-6, kernel="plain")
    b = oracle.log_weights(w.astype(np.int64))
    xf = oracle.xmatrix(b, 32.0, uf.cpu().numpy(), vf.cpu().numpy())
    xp = oracle.xmatrix(b, 32.0, up.cpu().numpy(), vp.cpu().numpy())
    assert np.max(np.abs(xf - xp)) < 8 * lg_err_bound(32.0)


def test_fp64_path_is_tight(ctx):
    w = W.uniform(200, 1, 30000, 78, dtype=np.int16)
    ps = [1.0, 4.0, 16.0, 64.0]
    d, u, v, info, b, uo, vo, swo, sto = run_both(ctx, w, ps, tol=1e-10, prec="fp64")
    assert info["status"] == 0 and sto == 0
    xg = oracle.xmatrix(b, 64.0, u, v)
    xo = oracle.xmatrix(b, 64.0, uo, vo)
    assert np.max(np.abs(xg - xo)) < 1e-8
    # same iteration, same stopping rule family: sweep counts agree within one per step
    r, c = oracle.sums(b, 64.0, u, v)
    assert np.abs(c - 1).max() < 1e-9


def test_precision_modes_order(ctx):
    """FP64-recomputed sums at p = 128: the FP64 path and the per-step matrix path (the
    default for MIXED) stay at the stopping tol; the single-read kernel's error grows with p
    as the FP32 logarithm bound says, and is the largest."""
    w = W.uniform(300, 1, 1000, 79, dtype=np.int16)
    ps = [2.0 ** k for k in range(8)]
    b = oracle.log_weights(w.astype(np.int64))
    errs = {}
    for name, prec, kernel in (("step", "mixed", "auto"), ("fused", "mixed", "fused"), ("fp32", "fp32", "auto"),
                               ("fp64", "fp64", "auto")):
        d = api.to_device(w)
        u, v, info = api.sa_scale(ctx, d, ps, 1e-6, prec=prec, kernel=kernel)
        r, c = oracle.sums(b, ps[-1], u.cpu().numpy(), v.cpu().numpy())
        errs[name] = max(np.abs(r - 1).max(), np.abs(c - 1).max())
    assert errs["fp64"] < 2e-6 and errs["step"] < 2e-6, errs
    assert errs["fused"] < 2 * lg_err_bound(ps[-1]) + 2e-6, errs
    assert max(errs["fp64"], errs["step"]) <= errs["fused"] + 1e-12, errs


def test_resume_equals_full_run(ctx):
    w = W.uniform(400, 1, 1000, 80, dtype=np.int16)
    ps = [1.0, 2.0, 4.0, 8.0, 16.0]
    d = api.to_device(w)
    u1, v1, _ = api.sa_scale(ctx, d, ps, 1e-6)
    u2, v2, _ = api.sa_scale(ctx, d, ps[:3], 1e-6)
    u3, v3, info = api.sa_scale(ctx, d, ps, 1e-6, resume_from=3, u=u2, v=v2)
    assert info["steps_done"] == 2
    b = oracle.log_weights(w.astype(np.int64))
    x1 = oracle.xmatrix(b, 16.0, u1.cpu().numpy(), v1.cpu().numpy())
    x3 = oracle.xmatrix(b, 16.0, u3.cpu().numpy(), v3.cpu().numpy())
    assert np.max(np.abs(x1 - x3)) < 8 * lg_err_bound(16.0)


def test_not_converged_and_nonfinite_status(ctx):
    w = W.uniform(256, 1, 1000, 81, dtype=np.int16)
    d = api.to_device(w)
    _, _, info = api.sa_scale(ctx, d, [1.0, 256.0], 1e-12, 3)
    assert info["status"] == api.SaError(-4, "").status and info["converged"] == 0
    w0 = w.copy()
    w0[17, :] = 0
    d0 = api.to_device(w0)
    for kernel in ("fused", "plain", "step"):
        with pytest.raises(api.SaError) as e:
            api.sa_scale(ctx, d0, [1.0, 2.0], 1e-6, 50, kernel=kernel)
        assert e.value.status == -6


def test_invalid_arguments_are_errors(ctx):
    w = W.uniform(64, 1, 1000, 82, dtype=np.int16)
    d = api.to_device(w)
    for bad in ([], [2.0, 1.0], [0.0], [1.0, float("nan")]):
        with pytest.raises((api.SaError, ValueError)):
            api.sa_scale(ctx, d, bad, 1e-6)
    with pytest.raises(api.SaError):
        api.sa_scale(ctx, d, [1.0], -1.0)
