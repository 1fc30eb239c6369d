"""The autotuner on the GPU: a short tuning run gives a valid plan, the library takes it,
the batch's results under it match the oracle, and a second call reads the cache."""
import numpy as np
import pytest

import oracle
from paper_1104_3830_gb300 import api
from paper_1104_3830_gb300 import autotune as A
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


def test_tune_cache_and_apply(ctx, tmp_path):
    cache = str(tmp_path / "plan.json")
    kw = dict(count_per_bucket=12, ps=[1.0, 2.0, 4.0], max_sweeps=2000, reps=1)
    plan, choice, src = A.load_or_tune(ctx, np.int16, cache=cache, **kw)
    assert src.startswith("tuned")
    assert set(choice) == {A.bucket_name(lo, hi) for lo, hi in A.BUCKETS}
    plan2, choice2, src2 = A.load_or_tune(ctx, np.int16, cache=cache, **kw)
    assert src2.startswith("cache") and choice2 == choice and plan2 == plan
    api.sa_set_batch_plan(ctx, plan)
    try:
        mats = [W.uniform(n, 1, 1000, 1400 + n, dtype=np.int16) for n in (10, 40, 90, 200, 400)]
        pack = A._Pack(mats)
        from paper_1104_3830_gb300 import _lib as L
        ps = [1.0, 2.0, 4.0]
        rc = pack.run(ctx, L.make_opts(ps, 1e-6, 20000))
        assert rc == 0
        u, v = pack.u.cpu().numpy(), pack.v.cpu().numpy()
        o = 0
        for m in mats:
            n = m.shape[0]
            b = oracle.log_weights(m.astype(np.int64))
            r, c = oracle.sums(b, ps[-1], u[o:o + n], v[o:o + n])
            assert max(np.abs(r - 1).max(), np.abs(c - 1).max()) < 2 * ps[-1] * np.log(2) * 1e-6 + 4e-6
            o += n
    finally:
        api.sa_set_batch_plan(ctx, None)
