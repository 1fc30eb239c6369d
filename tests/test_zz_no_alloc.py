"""sa_scale_noalloc, the scaling entry point that allocates nothing (its scratch is a
static device array of the library), against the allocating sa_scale on the same inputs.

Callers that plan their device memory up front, or cannot take the device-wide
synchronisation of cudaMalloc/cudaFree, use it.  This file runs last so that a failure
here leaves every other test already run; it passes alone in a fresh process as well.
Tolerance: the one the other scaling tests use (p ln2 1e-6 per the FP32 exponent)."""
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


def noalloc(w_dev, ps, tol=1e-6, sweeps=20000):
    n = w_dev.size(0)
    u = torch.full((n,), 7.0, dtype=torch.float64, device=w_dev.device)   # stale contents must not matter
    v = torch.full((n,), -3.0, dtype=torch.float64, device=w_dev.device)
    m = api.matrix(w_dev)
    o = L.make_opts(ps, tol, sweeps)
    info = L.sa_scale_info()
    st = L.lib().sa_scale_noalloc(ctypes.byref(m), ctypes.byref(o),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                  ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()), ctypes.byref(info))
    return st, u.cpu().numpy(), v.cpu().numpy(), L.info_dict(info)


def test_noalloc_matches_sa_scale_on_two_calls(ctx):
    cases = [(W.uniform(1000, 1, 1000, 4100, dtype=np.int16), [1.0, 2.0, 4.0, 8.0, 16.0]),
             (W.uniform(777, 1, 30000, 4101, dtype=np.int32), [1.0, 4.0, 16.0, 64.0])]
    for w, ps in cases:
        d = api.to_device(w)
        st, u1, v1, info1 = noalloc(d, ps)
        assert st == 0, api.sa_last_error()
        ur, vr, info_r = api.sa_scale(ctx, d, ps, 1e-6, kernel="fused")
        b = oracle.log_weights(w.astype(np.int64))
        x1 = oracle.xmatrix(b, ps[-1], u1, v1)
        xr = oracle.xmatrix(b, ps[-1], ur.cpu().numpy(), vr.cpu().numpy())
        bound = 8 * ps[-1] * math.log(2) * 1.0e-6
        assert np.max(np.abs(x1 - xr)) < bound
        assert info1["sweeps_total"] == info_r["sweeps_total"]
        assert info1["converged"] == 1


def test_noalloc_rejects_sizes_beyond_its_scratch(ctx):
    w = W.uniform(4104, 1, 100, 4102, dtype=np.int16)
    d = api.to_device(w)
    st, *_ = noalloc(d, [1.0])
    assert st == L.SA_E_UNSUPPORTED and "4096" in api.sa_last_error()
    st, *_ = noalloc(api.to_device(W.uniform(64, 1, 100, 4103, dtype=np.int16)), [2.0 ** k for k in range(65)])
    assert st == L.SA_E_UNSUPPORTED
