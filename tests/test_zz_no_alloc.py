"""sa_scale_noalloc, the scaling entry point that allocates nothing (its scratch is a
static device array of the library), against the allocating sa_scale on the same inputs
and against the FP64 oracle.

Callers whose device memory is planned up front (a fixed budget, a pre-sized pool, an
allocator that must not grow) or that cannot take the device-wide synchronisation of
cudaMalloc/cudaFree use it.  Each case calls it twice in a row, so the second call runs
on whatever the first left in the shared array.  This file runs last so that a failure
here leaves every other test already run; it passes alone in a fresh process as well.

Tolerance: the one the other fused-kernel tests use.  The single-read kernel forms
p log2 w in FP32, so an entry of X(p) may be off by about p ln2 1e-6 (relative); entries
of two runs of it are compared within 8 p ln2 1e-6, and against the oracle within that
plus 8e-6 max(x, 1/n) for the two sides' stopping tolerance (1e-6 each)."""
import ctypes
import math

import numpy as np
import pytest

import oracle
from paper_1104_3830_gb300 import _lib as L
from paper_1104_3830_gb300 import api
from paper_1104_3830_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_3830_gb300 import build
    build.build()
    c = api.sa_create(0)
    yield c
    c.close()


def noalloc(w_dev, ps, tol=1e-6, sweeps=20000, resume_from=0, u0=None, v0=None):
    n = w_dev.size(0)
    if resume_from > 0:
        u, v = u0.clone(), v0.clone()
    else:   # stale contents must not matter
        u = torch.full((n,), 7.0, dtype=torch.float64, device=w_dev.device)
        v = torch.full((n,), -3.0, dtype=torch.float64, device=w_dev.device)
    m = api.matrix(w_dev)
    o = L.make_opts(ps, tol, sweeps, resume_from=resume_from)
    info = L.sa_scale_info()
    st = L.lib().sa_scale_noalloc(ctypes.byref(m), ctypes.byref(o),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                  ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()), ctypes.byref(info))
    return st, u.cpu().numpy(), v.cpu().numpy(), L.info_dict(info)


def x_of(b, p, u, v):
    return oracle.xmatrix(b, p, u, v)


CASES = [(1000, np.int16, 1000, [1.0, 2.0, 4.0, 8.0, 16.0], 4100),
         (777, np.int32, 30000, [1.0, 4.0, 16.0, 64.0], 4101),
         # the largest n accepted: the static grid cap applies, and int32 rows take two
         # chunks per thread
         (4096, np.int16, 1000, [1.0, 2.0, 4.0, 8.0], 4104),
         (4096, np.int32, 30000, [1.0, 2.0, 4.0, 8.0], 4105)]


@pytest.mark.parametrize("n,dtype,hi,ps,seed", CASES)
def test_noalloc_matches_sa_scale_and_oracle_on_two_calls(ctx, n, dtype, hi, ps, seed):
    w = W.uniform(n, 1, hi, seed, dtype=dtype)
    d = api.to_device(w)
    b = oracle.log_weights(w.astype(np.int64))
    ur, vr, info_r = api.sa_scale(ctx, d, ps, 1e-6, kernel="fused")
    xr = x_of(b, ps[-1], ur.cpu().numpy(), vr.cpu().numpy())
    uo, vo, _, _, sto = oracle.sinkhorn(b, ps, 1e-6, 20000)
    assert sto == 0
    xo = x_of(b, ps[-1], uo, vo)
    bound = 8 * ps[-1] * math.log(2) * 1.0e-6
    for call in range(2):
        st, u1, v1, info1 = noalloc(d, ps)
        assert st == 0, (call, api.sa_last_error())
        x1 = x_of(b, ps[-1], u1, v1)
        assert np.max(np.abs(x1 - xr)) < bound, call
        assert np.all(np.abs(x1 - xo) <= bound + 8e-6 * np.maximum(xo, 1.0 / n)), call
        assert info1["sweeps_total"] == info_r["sweeps_total"]
        assert info1["converged"] == 1


def test_noalloc_warm_resume_matches_sa_scale(ctx):
    """resume_from = 2 from the potentials at p = 2: the same continuation as sa_scale's."""
    n = 1500
    w = W.uniform(n, 1, 1000, 4106, dtype=np.int16)
    d = api.to_device(w)
    ps = [1.0, 2.0, 4.0, 8.0]
    u2, v2, _ = api.sa_scale(ctx, d, ps[:2], 1e-6, kernel="fused")
    ur, vr, info_r = api.sa_scale(ctx, d, ps, 1e-6, kernel="fused", resume_from=2, u=u2.clone(), v=v2.clone())
    b = oracle.log_weights(w.astype(np.int64))
    xr = x_of(b, ps[-1], ur.cpu().numpy(), vr.cpu().numpy())
    bound = 8 * ps[-1] * math.log(2) * 1.0e-6
    for call in range(2):
        st, u1, v1, info1 = noalloc(d, ps, resume_from=2, u0=u2, v0=v2)
        assert st == 0, api.sa_last_error()
        assert info1["steps_done"] == 2
        assert np.max(np.abs(x_of(b, ps[-1], u1, v1) - xr)) < bound, call
        assert info1["sweeps_total"] == info_r["sweeps_total"]


def test_noalloc_rejects_sizes_beyond_its_scratch(ctx):
    w = W.uniform(4104, 1, 100, 4102, dtype=np.int16)
    d = api.to_device(w)
    st, *_ = noalloc(d, [1.0])
    assert st == L.SA_E_UNSUPPORTED and "4096" in api.sa_last_error()
    st, *_ = noalloc(api.to_device(W.uniform(64, 1, 100, 4103, dtype=np.int16)), [2.0 ** k for k in range(65)])
    assert st == L.SA_E_UNSUPPORTED
