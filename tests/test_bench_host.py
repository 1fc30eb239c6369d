"""Host-side pieces of bench.py (no GPU): the module imports, every name the JSON line
uses is defined, the traffic table is consistent, and the workloads have the stated
shapes."""
import importlib.util
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_bench_names_and_tables():
    b = _bench()
    assert set(b.KERNEL_NAMES) == {1, 2, 3, 4}
    per_sweep, src = b.measured_traffic(3, 8192, 2)
    # either the capture matches the current kernel source or the figure is withheld; DRAM
    # bytes per sweep stay below one read of K plus the column partials (about 280 MB; L2
    # serves part of K) and above nothing
    assert (per_sweep is None and src is None) or (0 < per_sweep < 285e6 and "ncu" in src)
    assert b.measured_traffic(1, 12345, 2) == (None, None)
    assert b.load_peaks()[0] > 0


def test_bench_workload_shapes():
    b = _bench()
    w, ps, cfg = b.workload("uniform256")
    assert w.shape == (256, 256) and w.dtype == np.int32 and ps[-1] == 256.0 and "workload" in cfg
    w, ps, cfg = b.workload("small")
    assert w.shape == (2048, 2048) and w.dtype == np.int16


def test_oracle_baselines_small():
    """The CPU-baseline legs on tiny inputs: finite rates, the stated units, and the oracle's
    Algorithm 1 result fields."""
    b = _bench()
    from paper_1104_3830_gb300 import workloads as W
    w = W.uniform(64, 1, 1000, 11, dtype=np.int16)
    cb = b.cpu_baseline(w, [1.0, 2.0], budget_s=0.2)
    assert cb["value"] > 0 and cb["unit"] == "sweeps/s" and cb["one_core"]["cores"] == 1
    assert "one_core" not in b.cpu_baseline(w, [1.0], budget_s=0.1, one_core=False)
    mats = [W.uniform(n, 1, 1000, 12 + n, dtype=np.int32) for n in (16, 23, 40)]
    ib = b.oracle_instances_baseline(mats, [1.0, 2.0, 4.0], budget_s=0.5)
    assert ib["unit"] == "instances/s" and ib["value"] > 0
    a1 = b.oracle_algorithm1_baseline(W.uniform(40, 1, 1000, 13, dtype=np.int32).astype(np.int64),
                                      opt_ratio=2.0, p0=100.0, dp=50.0, max_rounds=30)
    assert a1["unit"] == "ms" and a1["status"] == 0 and a1["gamma"] <= 2.0
