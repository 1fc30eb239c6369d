"""The continuous-batching server (sa_submit / sa_poll): results of a mixed stream equal
those of each request solved alone (exact optimum, same product), the budget is enforced,
and small requests join the device-resident queue's running kernel."""
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
    h, o = make_server(lib, 256 << 20, [1.0, 2.0])
    try:
        # n = 8192 is charged about 22 n^2 bytes (matrix, K, log2 pairs, reduced arrays):
        # over 256 MiB
        assert lib.sa_server_request_bytes(h, L.SA_I16, 8192) > 256 << 20
        big = W.uniform(8192, 1, 1000, 5, dtype=np.int16)
        st, _ = submit(lib, h, big)
        assert st == L.SA_E_BUDGET
        # n = 2000: about 90 MiB each, admitted a few at a time
        charge = lib.sa_server_request_bytes(h, L.SA_I16, 2000)
        assert 2000 * 2000 * 2 < charge < 256 << 20
        ok = W.uniform(2000, 1, 1000, 6, dtype=np.int16)
        ts = [submit(lib, h, ok)[1] for _ in range(12)]
        for t in ts:
            st, perm, r = wait(lib, h, t)
            assert st == 0 and sorted(perm) == list(range(2000))
    finally:
        lib.sa_server_destroy(h)


SERVER_CONSTANT = 64 << 20   # the workers' persistent state the budget does not cover


def test_device_use_stays_within_budget(lib):
    """A mixed stream under a budget that admits only a few large requests at a time: the
    device memory in use (cudaMemGetInfo, sampled every millisecond from another thread)
    never exceeds the idle server's by more than the budget plus SERVER_CONSTANT."""
    import threading
    ps = [2.0 ** k for k in range(5)]
    budget = 512 << 20
    sizes = [3000, 40, 2500, 100, 3000, 300, 2800, 64, 512, 2600, 900, 33, 3000, 2200]
    mats = [W.uniform(n, 1, 1000, 3100 + n, dtype=np.int16) for n in sizes]
    h, o = make_server(lib, budget, ps)
    try:
        # warm-up pass: modules loaded, workers' small workspaces at their size
        ts = [submit(lib, h, m)[1] for m in mats]
        for t in ts:
            assert wait(lib, h, t)[0] == 0
            lib.sa_result_release(h, t)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        low = [free0]
        stop = threading.Event()

        def sample():
            while not stop.is_set():
                low[0] = min(low[0], torch.cuda.mem_get_info()[0])
                time.sleep(0.001)
        th = threading.Thread(target=sample)
        th.start()
        try:
            ts = [submit(lib, h, m)[1] for m in mats]
            res = [wait(lib, h, t) for t in ts]
        finally:
            stop.set()
            th.join()
        for m, (st, perm, r) in zip(mats, res):
            assert st == 0 and sorted(perm) == list(range(m.shape[0]))
        used = free0 - low[0]
        assert used <= budget + SERVER_CONSTANT, (used >> 20, budget >> 20)
    finally:
        lib.sa_server_destroy(h)


def test_allocation_failure_fails_each_request(lib):
    """A device allocation that fails (injected on the host: the server's allocation call
    reports out-of-memory without allocating) finishes the request with SA_E_NOMEM, for a
    small request (batched path) and a large one (sa_assign path); later requests run."""
    h, o = make_server(lib, 1 << 30, [1.0, 2.0, 4.0])
    try:
        small = W.uniform(100, 1, 1000, 3201, dtype=np.int16)
        large = W.uniform(1000, 1, 1000, 3202, dtype=np.int16)
        for m in (small, large):
            lib.sa_debug_fail_allocs(1)
            try:
                st, t = submit(lib, h, m)
                assert st == 0
                st, perm, r = wait(lib, h, t)
            finally:
                lib.sa_debug_fail_allocs(0)
            assert st == L.SA_E_NOMEM and r.status == L.SA_E_NOMEM, (st, r.status)
            st, t = submit(lib, h, m)
            st, perm, r = wait(lib, h, t)
            assert st == 0
            b = oracle.log_weights(m.astype(np.int64))
            assert oracle.perm_weight_exact(m, perm) == oracle.perm_weight_exact(m, oracle.hungarian(b)[0])
    finally:
        lib.sa_server_destroy(h)


def stats(lib, h):
    st = L.sa_server_stats()
    L.check(lib.sa_server_get_stats(h, ctypes.byref(st)))
    return st


def test_small_requests_join_the_running_queue(lib):
    """Small requests published while the request queue's kernel is scaling a long one are
    taken by its idle blocks at once: each finishes before the long one, all on the same
    launch, with certified optima.  After the queue has been idle its kernel ends, and the
    next request starts it again."""
    ps = [2.0 ** k for k in range(15)]
    h, o = make_server(lib, 1 << 30, ps, sweeps=20000)
    try:
        # uniform weights on a wide range at p up to 2^14: thousands of sweeps per step
        slow = W.uniform(300, 1, 30000, 3300, dtype=np.int16)
        # equal row and column sums at every p: one sweep per step
        fast = []
        for n in (40, 64, 100, 200, 333):
            m = np.ones((n, n), dtype=np.int16)
            np.fill_diagonal(m, 1000)
            fast.append(m)
        st, t_slow = submit(lib, h, slow)
        assert st == 0
        t0 = time.time()
        while stats(lib, h).live_launches < 1:
            assert time.time() - t0 < 10
            time.sleep(0.001)
        time.sleep(0.005)
        tf = [submit(lib, h, m)[1] for m in fast]
        res_fast = [wait(lib, h, t) for t in tf]
        st_slow, perm_slow, r_slow = wait(lib, h, t_slow)
        assert st_slow == 0
        for m, (st, perm, r) in zip(fast, res_fast):
            assert st == 0
            assert np.array_equal(perm, np.arange(m.shape[0]))   # the heavy diagonal
            assert r.t_done < r_slow.t_done, (r.t_done, r_slow.t_done)
            assert r.t_start <= r.t_scaled <= r.t_done
        b = oracle.log_weights(slow.astype(np.int64))
        assert oracle.perm_weight_exact(slow, perm_slow) == oracle.perm_weight_exact(slow, oracle.hungarian(b)[0])
        s1 = stats(lib, h)
        assert s1.live_launches == 1, s1.live_launches
        assert s1.live_requests == 1 + len(fast)
        # idle: every block leaves; the next request launches the kernel again
        time.sleep(0.1)
        st, t = submit(lib, h, fast[0])
        assert wait(lib, h, t)[0] == 0
        s2 = stats(lib, h)
        assert s2.live_launches == 2 and s2.live_requests == 2 + len(fast)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        assert s2.live_device_bytes > 0 and 2 * s2.large_grid <= sms and s2.live_slots * s2.live_blocks <= sms
    finally:
        lib.sa_server_destroy(h)


def test_large_request_after_the_queue_went_idle(lib):
    """The request queue's launch takes every SM the large requests leave; once its
    requests are done and its kernel has left, a large request gets its full grid back
    (the SMs of an ended launch are counted free even when nothing else is in flight)."""
    ps = [2.0 ** k for k in range(5)]
    h, o = make_server(lib, 4 << 30, ps)
    try:
        small = [W.uniform(n, 1, 1000, 3400 + n, dtype=np.int16) for n in (50, 120, 300)]
        for t in [submit(lib, h, m)[1] for m in small]:
            assert wait(lib, h, t, timeout=60)[0] == 0
        time.sleep(0.05)   # the queue's kernel leaves after 2 ms without requests
        large = W.uniform(700, 1, 1000, 3410, dtype=np.int16)
        st, t = submit(lib, h, large)
        st, perm, r = wait(lib, h, t, timeout=60)
        assert st == 0
        b = oracle.log_weights(large.astype(np.int64))
        assert oracle.perm_weight_exact(large, perm) == oracle.perm_weight_exact(large, oracle.hungarian(b)[0])
    finally:
        lib.sa_server_destroy(h)
