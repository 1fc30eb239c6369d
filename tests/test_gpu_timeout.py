"""Failure detection without a GPU fault: every barrier and ring wait of the step kernel is
bounded, and a wait that runs out makes the kernel record SA_E_TIMEOUT, wait (up to 2 s)
for its own copies in flight and return.  The test makes one wait run out for certain: the
context's testing hook SA_OPT_TEST_UNREACHABLE_BARRIER makes the kernel's first grid
barrier wait for one arrival more than the grid has (a flag that nothing sets), and the
limit SA_OPT_WAIT_LIMIT_NS is shortened to 1 ms.  Nothing is broken and no wait is
removed.  The call must return SA_E_TIMEOUT, leave a warm start as it was given, and leave
the context usable: with the hook off and the default limit the same context then scales
the same matrix to the oracle's X(p)."""
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


def test_wait_limit_runs_out_and_context_recovers(ctx):
    n = 2048
    w = W.uniform(n, 1, 1000, 4200, dtype=np.int16)
    d = api.to_device(w)
    ps = [1.0, 2.0, 4.0]
    api.sa_set_option(ctx, "wait_limit_ns", 1_000_000)
    api.sa_set_option(ctx, "test_unreachable_barrier", 1)
    try:
        with pytest.raises(api.SaError) as e:
            api.sa_scale(ctx, d, ps, 1e-6, 2000, kernel="step")
        assert e.value.status == -8 and "timed out" in str(e.value), e.value
        # a warm start survives the failure bit for bit
        u0 = torch.linspace(-3.0, 5.0, n, dtype=torch.float64, device="cuda")
        v0 = torch.linspace(7.0, -1.0, n, dtype=torch.float64, device="cuda")
        u1, v1 = u0.clone(), v0.clone()
        with pytest.raises(api.SaError) as e:
            api.sa_scale(ctx, d, ps, 1e-6, 2000, kernel="step", resume_from=1, u=u1, v=v1)
        assert e.value.status == -8, e.value
        assert torch.equal(u1, u0) and torch.equal(v1, v0)
    finally:
        api.sa_set_option(ctx, "test_unreachable_barrier", 0)
        api.sa_set_option(ctx, "wait_limit_ns", 2_000_000_000)
    u, v, info = api.sa_scale(ctx, d, ps, 1e-6, 2000, kernel="step")
    assert info["status"] == 0 and info["kernel_used"] == 3, info
    b = oracle.log_weights(w.astype(np.int64))
    uo, vo, _, _, st = oracle.sinkhorn(b, ps, 1e-6, 2000)
    assert st == 0
    xg = oracle.xmatrix(b, ps[-1], u.cpu().numpy(), v.cpu().numpy())
    xo = oracle.xmatrix(b, ps[-1], uo, vo)
    assert np.all(np.abs(xg - xo) <= 8e-6 * np.maximum(xo, 1.0 / n) + 1e-9)


def test_option_values_are_checked(ctx):
    for name, bad in (("wait_limit_ns", -1), ("solve_gpu", 2), ("step_sparse", -1), ("fused_threads", 384),
                      ("max_grid", -5), ("step_l2_bytes", -1), ("test_unreachable_barrier", 3)):
        with pytest.raises(api.SaError) as e:
            api.sa_set_option(ctx, name, bad)
        assert e.value.status == -1
