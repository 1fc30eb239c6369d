"""The continuous-batching server (sa_submit / sa_poll): results of a mixed stream equal
those of each request solved alone (exact optimum, same product), and the budget is
enforced."""
import ctypes
import time

import numpy as np
import pytest

import oracle
from paper_1104_3830_gb300 import _lib as L
from paper_1104_3830_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1104_3830_gb300 import build
    build.build()
    return L.lib()


def make_server(lib, budget, ps, tol=1e-6, sweeps=3000, threads=2):
    o = L.make_opts(ps, tol, sweeps)
    h = ctypes.c_void_p()
    L.check(lib.sa_server_create(ctypes.byref(h), 0, ctypes.c_size_t(budget), ctypes.byref(o), threads))
    return h, o


def submit(lib, h, w):
    t = ctypes.c_uint64()
    wt = L.SA_I16 if w.dtype == np.int16 else L.SA_I32
    st = lib.sa_submit(h, ctypes.c_void_p(w.ctypes.data), wt, w.shape[0], ctypes.byref(t))
    return st, t.value


def wait(lib, h, ticket, timeout=120.0):
    r = L.sa_result()
    t0 = time.time()
    while True:
        st = lib.sa_poll(h, ticket, ctypes.byref(r))
        if st != L.SA_PENDING:
            perm = np.ctypeslib.as_array(r.perm, shape=(r.n,)).copy() if r.perm else None
            return st, perm, r
        assert time.time() - t0 < timeout
        time.sleep(0.002)


def test_mixed_stream_is_exact_and_matches_alone(lib):
    ps = [2.0 ** k for k in range(7)]
    sizes = [40, 700, 100, 1500, 33, 300, 2000, 64, 512, 900]
    mats = [W.uniform(n, 1, 1000, 3000 + n, dtype=np.int16) for n in sizes]
    h, o = make_server(lib, 4 << 30, ps)
    try:
        tickets = []
        for m in mats:
            st, t = submit(lib, h, m)
            assert st == 0
            tickets.append(t)
        mixed = [wait(lib, h, t) for t in tickets]
        # each request again, alone
        alone = []
        for m in mats:
            st, t = submit(lib, h, m)
            alone.append(wait(lib, h, t))
        for m, (st, perm, r), (st2, perm2, r2) in zip(mats, mixed, alone):
            assert st == 0 and st2 == 0
            b = oracle.log_weights(m.astype(np.int64))
            ref = oracle.perm_weight_exact(m, oracle.hungarian(b)[0])
            assert oracle.perm_weight_exact(m, perm) == ref
            assert oracle.perm_weight_exact(m, perm2) == ref
            assert r.t_done >= r.t_start >= r.t_submit
            # same program on the same input: identical sweeps alone and in the mix
            assert r.sweeps == r2.sweeps
    finally:
        lib.sa_server_destroy(h)


def test_budget_is_enforced(lib):
    h, o = make_server(lib, 64 << 20, [1.0, 2.0])
    try:
        big = W.uniform(8192, 1, 1000, 5, dtype=np.int16)   # 128 MiB > 64 MiB budget
        st, _ = submit(lib, h, big)
        assert st == L.SA_E_BUDGET
        ok = W.uniform(2000, 1, 1000, 6, dtype=np.int16)    # 8 MiB each: admitted a few at a time
        ts = [submit(lib, h, ok)[1] for _ in range(12)]
        for t in ts:
            st, perm, r = wait(lib, h, t)
            assert st == 0 and sorted(perm) == list(range(2000))
    finally:
        lib.sa_server_destroy(h)
