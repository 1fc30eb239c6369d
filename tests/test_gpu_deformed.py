"""The deformed Sinkhorn iteration (Sec. 3.2): one sweep at each p_m = a log(m + 1) of an
increasing sequence, with v carried from one p to the next (no rescaling).  Through the
C ABI it is a schedule with max_sweeps_per_p = 1 and warm_keep_v = 1; the oracle runs the
same iteration in FP64.  Both sides do the same 300 sweeps, so the iterates agree up to the
FP32 arithmetic of each kernel: for the single-read kernel its exponent error, about
ln2 * 1e-6 * p relative (p <= 23 here), for the step kernel about 2e-7 relative.
"""
import math

import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("kernel,tol_x,tol_c", [("fused", 1e-4, 5e-5), ("step", 1e-5, 5e-6)])
@pytest.mark.parametrize("n,dtype", [(64, np.int32), (130, np.int16)])
def test_deformed_iteration_matches_oracle(ctx, kernel, tol_x, tol_c, n, dtype):
    a = 4.0
    ps = [a * math.log(m + 1) for m in range(1, 301)]
    w = W.uniform(n, 1, 1000, 4242 + n, dtype=dtype)
    d = api.to_device(w)
    u, v, info = api.sa_scale(ctx, d, ps, 1e-12, 1, kernel=kernel, warm_keep_v=True)
    assert info["sweeps_total"] == len(ps)
    b = oracle.log_weights(w.astype(np.int64))
    uo, vo, sw, rs, st = oracle.sinkhorn(b, ps, 1e-12, 1, warm_keep_v=True)
    assert int(sw.sum()) == len(ps)
    xg = oracle.xmatrix(b, ps[-1], u.cpu().numpy(), v.cpu().numpy())
    xo = oracle.xmatrix(b, ps[-1], uo, vo)
    assert np.max(np.abs(xg - xo)) < tol_x, np.max(np.abs(xg - xo))
    # the iterate is column-stochastic after every sweep (the column update is last)
    c = xg.sum(axis=0)
    assert np.max(np.abs(c - 1.0)) < tol_c
