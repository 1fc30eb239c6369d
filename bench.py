#!/usr/bin/env python3
"""Benchmark of the Sinkhorn preprocessing hot path on GB300.

One step = one pass of the whole path over one instance: log-domain Sinkhorn over the
p schedule (the step kernel: one evaluation of the per-step FP32 matrix K per p, then one
read of K per sweep), prune + CSR compaction, exact solve of the reduced instance and the
LP-duality certificate on A (sa_assign).  The default workload is the planted n = 8192
instance (int16 weights, 128 MiB, p = 1, 2, ..., 512, tol 1e-6).

Prints one JSON line.  value = Sinkhorn sweeps per second over the whole step (all
ranks), roofline = the step kernel against the measured HBM copy bandwidth, e2e = the
same metric through sa_assign_host with the matrix in pinned host memory.  At one GPU the
line also carries the metric's two other parts, each timed in the same run with its own
clock record: "batched" (the 4096-instance batched form, instances/s of one persistent
launch against the plain one-instance-per-launch path, and a sample of exact optimal
weights against the oracle) and "serve" (the first requests of the Poisson stream through
the continuous-batching server against a plain FIFO path: p50/p99 latency, instances/s).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload planted8192|tied8192|uniform256|uniform20000|batch4096|serve|
                              precision20000|reduced|euclidean1000|small]

Under torchrun every rank runs its own replica on its own GPU (the instances are
independent: no collective on the data path); value sums the ranks' sweeps over the
max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Sinkhorn sweeps/s & % HBM peak; batched instances/s; serve p50/p99 vs plain"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM bytes per sweep (dram__bytes_read.sum + dram__bytes_write.sum from one ncu capture,
# divided by the sweeps of the captured launch), valid only for the kernel source the
# capture was taken on: after any change to these files the figure is unknown (null).
_TRAFFIC = {
    # step kernel: planted n=8192 int16, p=256 from a cold start, 200 sweeps + 1 evaluation of K
    (3, 8192, 2): ((37.355624e9 + 0.927293e9) / 200, "ncu capture, planted n=8192 int16, p=256, 200 sweeps (one launch)",
                   {"paper_1104_3830_gb300/csrc/sweep_step.cu":
                    "2714eb0a87182dc9e9501bed35d548eb3c7986a9c9daa6e21a14acfc754e8af6",
                    "paper_1104_3830_gb300/csrc/common.cuh":
                    "081ba7d34dae961c3679ac9acf1c076fd6b30bb4428eb03eabf3ad582049a6cc",
                    "paper_1104_3830_gb300/csrc/log2pair.cuh":
                    "d0d997e23dba7b51d1c07b556aa6d5e60d23cf230a79b17de392b2f3074ae3d0"}),
    # step kernel: uniform n=20000 int16, the whole p = 1..256 schedule (28 sweeps, 9 evaluations
    # of K) of one scaling call, per sweep
    (3, 20000, 2): ((69.183675e9 + 17.738929e9) / 28,
                    "ncu capture, uniform n=20000 int16, p=1..256, the whole call (28 sweeps, 9 evaluations of K)",
                    {"paper_1104_3830_gb300/csrc/sweep_step.cu":
                     "2714eb0a87182dc9e9501bed35d548eb3c7986a9c9daa6e21a14acfc754e8af6",
                     "paper_1104_3830_gb300/csrc/common.cuh":
                     "081ba7d34dae961c3679ac9acf1c076fd6b30bb4428eb03eabf3ad582049a6cc",
                     "paper_1104_3830_gb300/csrc/log2pair.cuh":
                     "d0d997e23dba7b51d1c07b556aa6d5e60d23cf230a79b17de392b2f3074ae3d0"}),
    # Newton solve kernel: planted n=8192 int16, the p = 1 step (19 operator applications)
    (4, 8192, 2): ((5.138667e9 + 0.108529e9) / 19,
                   "ncu capture, planted n=8192 int16, p = 1 step, 19 operator applications (one launch)",
                   {"paper_1104_3830_gb300/csrc/newton.cu":
                    "c2eec455daed25f172d2ae73ca4d2601943251565cbffcd0677bd4561ae59e10",
                    "paper_1104_3830_gb300/csrc/common.cuh":
                    "a6671f98cbd36384cd1797923d09a590dde55eb3479341ec323ebc1b9836442c",
                    "paper_1104_3830_gb300/csrc/log2pair.cuh":
                    "d0d997e23dba7b51d1c07b556aa6d5e60d23cf230a79b17de392b2f3074ae3d0"}),
}


KERNEL_NAMES = {1: "fused_kernel (single-read persistent sweep, SFU exp2/log2 per element)",
                2: "row_lse_kernel + col_partial_kernel (plain sweep, host loop)",
                3: "step_kernel (persistent sweep over the per-step FP32 matrix)",
                4: "nt_solve_kernel (persistent Newton-CG over the per-step FP32 matrix, one read per operator application)"}


def over_ranks(ms, units, dist=None, device="cpu"):
    """Whole-job timing of replicas: (the slowest rank's time, the units of all ranks).
    dist is torch.distributed with an initialised process group, or None for one rank."""
    if dist is None:
        return float(ms), float(units)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


def measured_traffic(kernel_used, n, wbytes):
    """(bytes per sweep, source) if a capture of this kernel source and size exists."""
    import hashlib
    ent = _TRAFFIC.get((kernel_used, n, wbytes))
    if ent is None:
        return None, None
    per_sweep, source, files = ent
    for rel, want in files.items():
        with open(os.path.join(ROOT, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != want:
                return None, None
    return per_sweep, source


def workload(name):
    from paper_1104_3830_gb300 import workloads as W
    if name == "planted8192":
        w, ps, pi, _ = W.c2()
        return w, ps, {"workload": "planted n=8192 int16 w<=10000, p=1..512 (x2), tol 1e-6"}
    if name == "tied8192":
        w, ps, pi, _ = W.c2(tied_frac=0.01)
        return w, ps, {"workload": "planted n=8192 int16, 1% tied pairs, p=1..512 (x2), tol 1e-6"}
    if name == "uniform256":
        w, ps = W.c1()
        return w, ps, {"workload": "uniform n=256 int32 w in [1,1000], p=1..256 (x2), tol 1e-6"}
    if name == "uniform20000":
        w, ps = W.c3()
        return w, ps, {"workload": "uniform n=20000 int16 w in [1,32767], p=1..256 (x2), tol 1e-6"}
    if name == "profile8192":
        w, ps, pi, _ = W.c2()
        return w, ps[:2], {"workload": "planted n=8192 int16, p=1,2 only (profiling case)"}
    if name == "profile8192p256":
        w, ps, pi, _ = W.c2()
        return w, [256.0], {"workload": "planted n=8192 int16, p=256 from a cold start (profiling case; "
                                        "use --max-sweeps to fix the sweep count)"}
    if name == "small":
        w = W.uniform(2048, 1, 10000, 5, dtype=np.int16)
        return w, [2.0 ** k for k in range(8)], {"workload": "uniform n=2048 int16 (profiling case)"}
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 6:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, val in zip(names, parts[2:6]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(w, ps, budget_s=12.0, one_core=True):
    """The FP64 oracle (as it stands) on this host: sweeps/s of its log-domain Sinkhorn on
    the same matrix, timed on a bounded number of sweeps at the top of the schedule."""
    import oracle
    b = oracle.log_weights(w.astype(np.int64))
    n = w.shape[0]
    p = float(ps[-1])
    u = np.zeros(n)
    v = np.zeros(n)
    cores = oracle.num_threads()      # loads (and if needed builds) the oracle first
    # one probe sweep, then as many as fit the budget
    t0 = time.perf_counter()
    u, v, s, r, st = oracle.sinkhorn_from(b, p, u, v, 1e-300, 1)
    one = max(time.perf_counter() - t0, 1e-6)
    k = max(1, min(200, int(budget_s / one)))
    t0 = time.perf_counter()
    oracle.sinkhorn_from(b, p, u, v, 1e-300, k)
    dt = time.perf_counter() - t0
    line = {"value": k / dt, "unit": "sweeps/s", "cores": cores, "kind": "oracle",
            "sample": f"{k} FP64 log-domain Sinkhorn sweeps of the oracle at p={p:g} on the same n={n} matrix"}
    if not one_core:
        return line
    # the same sweeps on one core, on a smaller sample (a probe sweep, then what fits)
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.sinkhorn_from(b, p, u, v, 1e-300, 1)
        one1 = max(time.perf_counter() - t0, 1e-6)
        k1 = max(1, min(50, int(budget_s / 2 / one1)))
        t0 = time.perf_counter()
        oracle.sinkhorn_from(b, p, u, v, 1e-300, k1)
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    line["one_core"] = {"value": k1 / dt1, "unit": "sweeps/s", "cores": 1,
                        "sample": f"{k1} sweeps of the same iteration on one thread"}
    return line


def oracle_instances_baseline(mats, ps, budget_s=10.0, tol=1e-6, max_sweeps=20000):
    """The oracle's FP64 Sinkhorn over the whole schedule, instance after instance in the
    workload's own (random) order until the budget is spent: instances/s on this host."""
    import oracle
    cores = oracle.num_threads()
    done, sweeps = 0, 0
    t0 = time.perf_counter()
    for m in mats:
        _, _, sw, _, _ = oracle.sinkhorn(oracle.log_weights(np.asarray(m, dtype=np.int64)), ps, tol, max_sweeps)
        done += 1
        sweeps += int(sw.sum())
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "instances/s", "cores": cores, "kind": "oracle",
            "sample": f"the first {done} instances of the workload, whole schedule to tol {tol:g} "
                      f"({sweeps} FP64 sweeps)"}


def oracle_algorithm1_baseline(w, **kw):
    """The oracle's Algorithm 1 (FP64 Sinkhorn, prune, exact solve of B) on the same matrix
    and settings: its wall time and result."""
    import oracle
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    r = oracle.algorithm1(w, **kw)
    dt = time.perf_counter() - t0
    return {"value": dt * 1e3, "unit": "ms", "cores": cores, "kind": "oracle",
            "sample": "the whole Algorithm 1 run on the same matrix", "gamma": r["gamma"],
            "p_final": r["p_final"], "rounds": r["rounds"], "sweeps": r["sweeps"], "status": r["status"]}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, ps, cfg = workload(args.workload)
    import oracle
    b = oracle.log_weights(w.astype(np.int64))
    n = w.shape[0]
    p = float(ps[-1])
    u = np.zeros(n)
    v = np.zeros(n)
    per_step = 2
    for _ in range(args.warmup):
        u, v, *_ = oracle.sinkhorn_from(b, p, u, v, 1e-300, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        u, v, *_ = oracle.sinkhorn_from(b, p, u, v, 1e-300, per_step)
    dt = time.perf_counter() - t0
    val = args.steps * per_step / dt
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "sweeps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(cfg, sample=f"{per_step} oracle sweeps at p={p:g} per step"),
            "cpu_baseline": {"value": val, "unit": "sweeps/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"{per_step} FP64 sweeps per step at p={p:g}, n={n}"},
            "e2e": {"value": val, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def certified_weight(ctx, d, p, u, v, max_repairs=64):
    """The exact optimum of one scaled instance from its potentials, as sa_assign finds it:
    prune (t = 1/n, row and column maxima kept), solve B toward v/p, certify on all of A
    and re-solve with the violating entries added.  Returns (perm, certified)."""
    from paper_1104_3830_gb300 import api
    n = d.size(0)
    rp, col, wv, _ = api.sa_prune(ctx, d, p, u, v)
    vv = v.cpu().numpy() / p
    perm, _, al, be = api.sa_solve_reduced(rp, col, wv, near=vv)
    for _ in range(max_repairs):
        nv, (arp, acol, aw) = api.sa_certify(ctx, d, al, be)
        if nv == 0:
            return perm, True
        rows = np.concatenate([np.repeat(np.arange(n), np.diff(rp)), np.repeat(np.arange(n), np.diff(arp))])
        cols = np.concatenate([col, acol])
        ws = np.concatenate([wv, aw])
        key = rows.astype(np.int64) * n + cols
        key, first = np.unique(key, return_index=True)
        rows, cols, ws = key // n, (key % n).astype(np.int32), ws[first]
        rp = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))]).astype(np.int64)
        col, wv = cols, ws.astype(np.int32)
        perm, _, al, be = api.sa_solve_reduced(rp, col, wv, beta0=be)
    return perm, False


def batched_part(args):
    """Batched form: 4096 independent dense instances, n log-uniform in [16, 512], int32
    weights in [1, 1000], p = 1, 2, ..., 128, scaled by sa_batch_scale under the
    autotuner's launch plan (one persistent launch per size bucket).  Beside it: the plain one-instance-per-launch path (plain and fused
    kernels) on a sample, and, for another sample, the certified optimum reached from the
    batch's potentials against the oracle's Hungarian optimum (exact integer products)."""
    import ctypes
    import torch
    import oracle
    from paper_1104_3830_gb300 import _lib as L
    from paper_1104_3830_gb300 import api
    from paper_1104_3830_gb300 import workloads as W
    mats, ps = W.c4(count=args.batch_count)
    k = len(mats)
    ns = np.array([m.shape[0] for m in mats], dtype=np.int32)
    lds = ((ns + 3) // 4 * 4).astype(np.int64)   # 16-byte pitch for int32
    offs_w = np.concatenate([[0], np.cumsum(lds * ns)[:-1]]).astype(np.int64)
    flat = np.zeros(int((lds * ns).sum()), dtype=np.int32)
    for m, o_, l_ in zip(mats, offs_w, lds):
        n = m.shape[0]
        flat[o_:o_ + n * l_].reshape(n, l_)[:, :n] = m
    dev = torch.from_numpy(flat).cuda()
    base = dev.data_ptr()
    ptrs = torch.tensor([base + 4 * int(o_) for o_ in offs_w], dtype=torch.int64, device="cuda")
    dn = torch.from_numpy(ns).cuda()
    dld = torch.from_numpy(lds).cuda()
    offs_np = np.concatenate([[0], np.cumsum(ns)[:-1]]).astype(np.int64)
    offs = torch.from_numpy(offs_np).cuda()
    tot = int(ns.sum())
    u = torch.zeros(tot, dtype=torch.float64, device="cuda")
    v = torch.zeros(tot, dtype=torch.float64, device="cuda")
    sw = np.zeros(k, dtype=np.int32)
    st = np.zeros(k, dtype=np.int32)
    o = L.make_opts(ps, 1e-6, args.max_sweeps)
    stream = torch.cuda.current_stream()
    ctx = api.sa_create(0, stream.cuda_stream)
    # the launch plan of the size buckets: the autotuner's cached choice for this GPU and
    # weight type, or a fresh tuning run (outside the timed region)
    from paper_1104_3830_gb300 import autotune
    plan, choice, plan_src = autotune.load_or_tune(ctx, np.int32)
    api.sa_set_batch_plan(ctx, plan)

    def once():
        return L.lib().sa_batch_scale(ctx.handle, k, ctypes.c_void_p(ptrs.data_ptr()), ctypes.c_void_p(dn.data_ptr()),
                                      ctypes.c_void_p(dld.data_ptr()), ctypes.c_void_p(offs.data_ptr()), L.SA_I32,
                                      ctypes.byref(o), ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                      sw.ctypes.data_as(L._I32P), st.ctypes.data_as(L._I32P))
    for _ in range(max(1, args.batch_warmup)):
        once()
    times = []
    launches0 = L.lib().sa_kernel_launches()
    with ClockSampler(0) as clk:
        for _ in range(args.batch_steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = once()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    launches = (L.lib().sa_kernel_launches() - launches0) // args.batch_steps
    ms = statistics.mean(times)
    value = k / (ms / 1e3)
    sweeps = int(sw.sum())
    elems = float(sum(int(n) * int(n) * int(s_) for n, s_ in zip(ns, sw)))
    # plain path: one instance per launch sequence (plain or fused kernels), on a sample
    rng = np.random.default_rng(0)
    sample = rng.choice(k, size=min(args.plain_sample, k), replace=False)
    plain = {}
    for kern in ("plain", "fused"):
        t0 = time.perf_counter()
        for q in sample:
            d = api.to_device(mats[q])
            api.sa_scale(ctx, d, ps, 1e-6, args.max_sweeps, kernel=kern)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        plain[kern] = len(sample) / dt if len(sample) else None
    # exact optimal weights of a sample, from the batch's potentials, against the oracle
    chk = rng.choice(k, size=min(args.check_sample, k), replace=False)
    equal = certified = 0
    for q in chk:
        n = int(ns[q])
        d = api.to_device(mats[q])
        uq = u[int(offs_np[q]):int(offs_np[q]) + n].clone()
        vq = v[int(offs_np[q]):int(offs_np[q]) + n].clone()
        perm, cert = certified_weight(ctx, d, ps[-1], uq, vq)
        b = oracle.log_weights(mats[q].astype(np.int64))
        ref = oracle.hungarian(b)[0]
        certified += int(cert)
        equal += int(oracle.perm_weight_exact(mats[q], perm) == oracle.perm_weight_exact(mats[q], ref))
    # SFU roofline: one ex2 per element per sweep (log2 tables in shared memory)
    ex2_peak = 30.0 * 152 * 2.07e9 / 1e12   # measured ex2/clk/SM x SMs x max clock (Tex2/s)
    achieved = elems / (ms / 1e3) / 1e12
    ctx.close()
    return {"value": value, "unit": "instances/s", "ms_per_launch": ms, "launches_timed": len(times),
            "workload": f"{k} instances, n log-uniform [16,512], int32 w in [1,1000], p=1..128 (x2), tol 1e-6",
            "impl": "sa_batch_scale (one persistent launch per size bucket, buckets side by side)",
            "plan": {"buckets": [list(x) for x in plan], "source": plan_src},
            "status_counts": {str(s_): int((st == s_).sum()) for s_ in np.unique(st)},
            "sweeps_total": sweeps, "l2": "instances re-read from L2/smem (working set < L2)",
            "plain_one_instance_per_launch": {"instances_per_s_plain_kernels": plain["plain"],
                                              "instances_per_s_fused_kernel": plain["fused"],
                                              "sample": len(sample)},
            "exact_check": {"sample": len(chk), "optimum_equal_to_oracle": equal, "certified": certified,
                            "how": "prune + exact solve + LP certificate from the batch's potentials, "
                                   "exact integer product against the oracle's Hungarian optimum"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": ex2_peak, "unit": "Tex2/s",
                         "frac": achieved / ex2_peak, "traffic": None,
                         "peak_source": "own micro-benchmark: 30 ex2/clk/SM x 152 SMs x 2.07 GHz"},
            "gpu_launches": int(launches), "clocks": clk.summary()}


def run_batch(args):
    """The batched form on its own line (value = instances/s of the persistent launch)."""
    import __graft_entry__
    __graft_entry__.build()
    part = batched_part(args)
    line = {"metric": METRIC, "value": part["value"], "unit": "instances/s", "n_gpus": 1,
            "steps": args.batch_steps, "warmup": args.batch_warmup, "ms_per_step": part["ms_per_launch"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (exp/sum), f64 potentials", "data": "synthetic",
            "config": {"workload": part["workload"], "status_counts": part["status_counts"],
                       "sweeps_total": part["sweeps_total"], "impl": part["impl"], "l2": part["l2"]},
            "plain_one_instance_per_launch": part["plain_one_instance_per_launch"],
            "exact_check": part["exact_check"], "roofline": part["roofline"],
            "gpu_launches": part["gpu_launches"], "clocks": part["clocks"]}
    if not args.no_cpu_baseline:
        from paper_1104_3830_gb300 import workloads as W
        mats, ps = W.c4(count=args.batch_count)
        line["cpu_baseline"] = oracle_instances_baseline(mats, ps)
    print(json.dumps(line), flush=True)


def run_precision(args):
    """Precision form: the dense n = 20000 int16 instance (weights uniform in [1, 32767],
    p = 1, 2, ..., 256) scaled by the mixed-precision path (per-step FP32 matrix, FP64
    potentials), the all-FP32 path (FP32 potentials) and the all-FP64 path on the same input;
    sweeps/s of the scaling and the error of each result against the FP64 oracle run on the
    same schedule: the largest deviation of an entry of X(p) from the oracle's (relative to
    max(x, 1/n)), the largest deviation of u_i + v_j on the entries with x > 1e-3, and the
    FP64 row and column sums of X(p) computed by the oracle from each path's potentials."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import oracle
    from paper_1104_3830_gb300 import _lib as L
    from paper_1104_3830_gb300 import api
    from paper_1104_3830_gb300 import workloads as W
    w, ps = W.c3()
    n = w.shape[0]
    stream = torch.cuda.current_stream()
    ctx = api.sa_create(0, stream.cuda_stream)
    d = api.to_device(w)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    launches0 = L.lib().sa_kernel_launches()
    paths, pots = {}, {}
    with ClockSampler(0) as clk:
        for name, prec in (("mixed", "mixed"), ("fp32", "fp32"), ("fp64", "fp64")):
            reps = 1 if prec == "fp64" else max(1, args.steps)
            for _ in range(1 if prec == "fp64" else args.warmup):
                api.sa_scale(ctx, d, ps, 1e-6, args.max_sweeps, prec=prec)
            times, infos = [], []
            for _ in range(reps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                u, v, info = api.sa_scale(ctx, d, ps, 1e-6, args.max_sweeps, prec=prec)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
                infos.append(info)
            info = infos[-1]
            pots[name] = (u.cpu().numpy(), v.cpu().numpy())
            ms = statistics.mean(times)
            paths[name] = {"sweeps": int(info["sweeps_total"]), "ms": ms,
                           "sweeps_per_s": info["sweeps_total"] / (ms / 1e3),
                           "kernel": KERNEL_NAMES.get(info["kernel_used"], "?"), "kernel_used": int(info["kernel_used"]),
                           "kernel_ms": info["kernel_ms"], "converged": int(info["converged"])}
    launches = L.lib().sa_kernel_launches() - launches0
    del d, flush
    # the FP64 oracle on the same schedule, then each path's error against it
    b = oracle.log_weights(w.astype(np.int64))
    t0 = time.perf_counter()
    uo, vo, swo, rso, sto = oracle.sinkhorn(b, ps, 1e-6, args.max_sweeps)
    oracle_s = time.perf_counter() - t0
    p = ps[-1]
    for name, (u, v) in pots.items():
        r, c = oracle.sums(b, p, u, v)
        xdev, sdev = 0.0, 0.0
        for r0 in range(0, n, 500):
            bb = p * b[r0:r0 + 500]
            xg = np.exp(bb - u[r0:r0 + 500, None] - v[None, :])
            xo = np.exp(bb - uo[r0:r0 + 500, None] - vo[None, :])
            xdev = max(xdev, float(np.max(np.abs(xg - xo) / np.maximum(xo, 1.0 / n))))
            big = xo > 1e-3
            if big.any():
                sg = (u[r0:r0 + 500, None] + v[None, :])[big]
                so = (uo[r0:r0 + 500, None] + vo[None, :])[big]
                sdev = max(sdev, float(np.max(np.abs(sg - so))))
        paths[name].update({"x_rel_err_vs_oracle": xdev, "u_plus_v_err_vs_oracle": sdev,
                            "fp64_row_sum_err": float(np.abs(r - 1).max()),
                            "fp64_col_sum_err": float(np.abs(c - 1).max())})
    peak, peak_kind = load_peaks()
    m = paths["mixed"]
    achieved = m["sweeps"] * n * n * 2 / (m["ms"] / 1e3) / 1e9
    # DRAM bytes per sweep of the whole call (evaluations of K included), when a capture of
    # this kernel source exists
    traffic, traffic_src = measured_traffic(m["kernel_used"], n, w.dtype.itemsize)
    line = {"metric": METRIC, "value": m["sweeps_per_s"], "unit": "sweeps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": m["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (exp/sum), f64 potentials", "data": "synthetic",
            "config": {"workload": "uniform n=20000 int16 w in [1,32767], p=1..256 (x2), tol 1e-6, scaling only "
                                   "(mixed / all-FP32 / all-FP64 paths on the same input)",
                       "l2": "flushed before every timed run (256 MiB write); the matrix (800 MB) exceeds L2"},
            "paths": paths,
            "oracle": {"sweeps": int(swo.sum()), "status": int(sto), "seconds": oracle_s, "cores": oracle.num_threads(),
                       "how": "FP64 log-domain Sinkhorn of the oracle on the same matrix and schedule"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "traffic_source": traffic_src or "none for this kernel source or size",
                         "kernel": m["kernel"], "peak_source": f"{peak_kind} hbm_gbs",
                         "note": "whole scaling call incl. the per-step evaluation of K, about 3 sweeps per step"},
            "e2e": None, "gpu_launches": int(launches), "clocks": clk.summary()}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = {"value": int(swo.sum()) / oracle_s, "unit": "sweeps/s", "cores": oracle.num_threads(),
                                "kind": "oracle", "sample": "the oracle's whole schedule on the same matrix "
                                                            "(the error reference above), sweeps per second"}
    print(json.dumps(line), flush=True)
    ctx.close()


def serve_part(args):
    """Serving form: the first requests of a Poisson stream of dense instances (n log-uniform
    in [32, 4096]) through the continuous-batching server (sa_submit/sa_poll), and the same
    requests at the same arrival times through a plain FIFO one-at-a-time path (sa_assign_host
    on the plain kernels); p50/p99 latency and instances/s of both."""
    import ctypes
    from paper_1104_3830_gb300 import _lib as L
    from paper_1104_3830_gb300 import api
    from paper_1104_3830_gb300 import workloads as W
    seed = W.BASE_SEED + 4
    pool_n = W.loguniform_sizes(args.serve_pool, 32, 4096, seed)
    pool = [W.c5_request(seed, q, int(n), args.serve_dist) for q, n in enumerate(pool_n)]
    arrivals = W.poisson_arrivals(args.serve_rate, args.serve_seconds, seed)[: args.serve_requests]
    ps = [2.0 ** q for q in range(9)]
    o = L.make_opts(ps, 1e-6, args.max_sweeps)
    lib = L.lib()

    def serve_run(arr):
        h = ctypes.c_void_p()
        L.check(lib.sa_server_create(ctypes.byref(h), 0, ctypes.c_size_t(40 << 30), ctypes.byref(o), 2))
        tickets = []
        t0 = time.perf_counter()
        for q, ta in enumerate(arr):
            while time.perf_counter() - t0 < ta:
                time.sleep(0.0002)
            m = pool[q % len(pool)]
            t = ctypes.c_uint64()
            L.check(lib.sa_submit(h, ctypes.c_void_p(m.ctypes.data), L.SA_I16, m.shape[0], ctypes.byref(t)))
            tickets.append(t.value)
        lat, done_t, first, bad, small, wait_adm, to_scaled = [], [], None, 0, [], [], []
        r = L.sa_result()
        deadline = time.perf_counter() + 600.0
        for t in tickets:
            while True:
                stt = lib.sa_poll(h, t, ctypes.byref(r))
                if stt != L.SA_PENDING:
                    break
                if time.perf_counter() > deadline:
                    raise RuntimeError(f"serve: request {t} still pending after 600 s")
                time.sleep(0.0005)
            bad += int(stt != 0)
            lat.append(r.t_done - r.t_submit)
            wait_adm.append(r.t_start - r.t_submit)
            to_scaled.append(r.t_scaled - r.t_submit if r.t_scaled > 0 else np.nan)
            small.append(r.n <= 512)
            done_t.append(r.t_done)
            first = r.t_submit if first is None else min(first, r.t_submit)
            lib.sa_result_release(h, t)
        stats = L.sa_server_stats()
        L.check(lib.sa_server_get_stats(h, ctypes.byref(stats)))
        lib.sa_server_destroy(h)
        lat = np.array(lat)
        small = np.array(small)
        wait_adm = np.array(wait_adm)
        to_scaled = np.array(to_scaled)
        span = max(done_t) - first

        def pct(x, w, sc=None):
            if not len(x):
                return None
            d = {"p50_ms": float(np.percentile(x, 50) * 1e3), "p99_ms": float(np.percentile(x, 99) * 1e3),
                 "admission_wait_p50_ms": float(np.percentile(w, 50) * 1e3), "requests": int(len(x))}
            if sc is not None and np.isfinite(sc).any():
                d["scaled_after_p50_ms"] = float(np.nanpercentile(sc, 50) * 1e3)
            return d
        return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "instances_per_s": len(lat) / span, "requests": len(lat), "failed": bad,
                "small_n_le_512": pct(lat[small], wait_adm[small], to_scaled[small]),
                "large": pct(lat[~small], wait_adm[~small]),
                "request_queue": {"launches": int(stats.live_launches), "requests": int(stats.live_requests),
                                  "blocks_per_launch": int(stats.live_blocks), "launch_slots": int(stats.live_slots),
                                  "large_grid": int(stats.large_grid)}}

    with ClockSampler(0) as clk:
        ours = serve_run(arrivals)
        # plain FIFO: one request at a time on the plain kernels, the same arrivals
        ctx = api.sa_create(0)
        lat, small = [], []
        t0 = time.perf_counter()
        for q, ta in enumerate(arrivals):
            now = time.perf_counter() - t0
            if now < ta:
                time.sleep(ta - now)
            m = pool[q % len(pool)]
            api.sa_assign_host(ctx, m, ps, 1e-6, args.max_sweeps, kernel="plain")
            lat.append(time.perf_counter() - t0 - ta)
            small.append(m.shape[0] <= 512)
        span = time.perf_counter() - t0 - arrivals[0]
        ctx.close()
    lat = np.array(lat)
    small = np.array(small)
    fifo = {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "instances_per_s": len(lat) / span, "requests": len(lat),
            "small_n_le_512": {"p50_ms": float(np.percentile(lat[small], 50) * 1e3),
                               "p99_ms": float(np.percentile(lat[small], 99) * 1e3), "requests": int(small.sum())}
            if small.any() else None}
    return {"value": ours["instances_per_s"], "unit": "instances/s",
            "workload": f"first {len(arrivals)} requests of a Poisson {args.serve_rate:g}/s stream, "
                        f"n log-uniform [32,4096], {args.serve_dist} weights, 40 GB budget, p=1..256 (x2); "
                        "the same requests and arrival times for both systems",
            "offered_per_s": args.serve_rate, "pool": len(pool), "serve": ours, "plain_fifo": fifo,
            "clocks": clk.summary()}


def run_serve(args):
    """The serving form on its own line (value = the server's instances/s)."""
    import __graft_entry__
    __graft_entry__.build()
    part = serve_part(args)
    line = {"metric": METRIC, "value": part["value"], "unit": "instances/s", "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 (exp/sum), f64 potentials", "data": "synthetic",
            "config": {"workload": part["workload"], "offered_per_s": part["offered_per_s"], "pool": part["pool"]},
            "serve": part["serve"], "plain_fifo": part["plain_fifo"], "clocks": part["clocks"]}
    print(json.dumps(line), flush=True)


def run_reduced(args):
    """Reduced-solve form: B from the scaling (p = 1, 2, ..., 256) and prune (t = 1/n) of
    uniform int16 instances (weights in [1, 1000], the serving distribution), solved exactly
    by the host solver from the column minima, from the scaling's duals, and from the
    column minima with the duals then moved next to the scaling's (sa_solve_reduced_near,
    as sa_assign solves B), and by the GPU path (sa_solve_reduced_gpu:
    GPU auction for the starting prices, host greedy pass and row reduction, each shortest
    augmenting path search on the GPU); wall time of each solve and the optimum (equal)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3830_gb300 import api
    from paper_1104_3830_gb300 import workloads as W
    ctx = api.sa_create(0, torch.cuda.current_stream().cuda_stream)
    ps = [2.0 ** k for k in range(9)]
    out = []
    for n in [int(x) for x in args.reduced_sizes.split(",")]:
        w = W.uniform(n, 1, 1000, 20261202 + 40 + n, dtype=np.int16)
        d = api.to_device(w)
        u, v, info = api.sa_scale(ctx, d, ps, 1e-6, 20000)
        rp, col, wv, _ = api.sa_prune(ctx, d, ps[-1], u, v)
        vv = v.cpu().numpy() / ps[-1]
        api.sa_solve_reduced_gpu(ctx, rp, col, wv, price0=vv)   # warm-up (build, allocation)
        tn = time.perf_counter()
        _, s_n, _, _ = api.sa_solve_reduced(rp, col, wv, near=vv)      # host, sa_assign's way
        tw = time.perf_counter()
        _, s_w, _, _ = api.sa_solve_reduced(rp, col, wv, beta0=vv)     # host, from the scaling's duals
        t0 = time.perf_counter()
        perm_h, s_h, _, _ = api.sa_solve_reduced(rp, col, wv)           # host, from the column minima
        t1 = time.perf_counter()
        perm_g, s_g, _, _, ai = api.sa_solve_reduced_gpu(ctx, rp, col, wv, price0=vv)
        t2 = time.perf_counter()
        # the oracle's dense Hungarian method on the same B (forbidden entries -inf), timed
        # beside as the CPU baseline of this line
        import oracle
        rows = np.repeat(np.arange(n), np.diff(rp))
        bb = np.full((n, n), -np.inf)
        bb[rows, col] = np.log(wv.astype(np.float64))
        t3 = time.perf_counter()
        ph, _, _, st = oracle.hungarian(bb)
        t4 = time.perf_counter()
        s_o = float(bb[np.arange(n), ph].sum()) if st == 0 else float("nan")
        out.append({"n": n, "nnz": int(len(col)), "host_ms": (t1 - t0) * 1e3, "host_warm_ms": (t0 - tw) * 1e3,
                    "host_near_ms": (tw - tn) * 1e3, "near_same_optimum": abs(s_n - s_h) <= 1e-9 + 1e-13 * abs(s_h),
                    "warm_same_optimum": abs(s_w - s_h) <= 1e-9 + 1e-13 * abs(s_h), "gpu_auction_ms": ai["auction_ms"],
                    "gpu_exact_phase_ms": ai["host_ms"], "gpu_total_ms": (t2 - t1) * 1e3,
                    "rounds": ai["rounds"], "phases": ai["phases"], "complete": ai["complete"],
                    "gpu_searches": ai["searches"], "gpu_search_rounds": ai["search_rounds"],
                    "same_optimum": abs(s_h - s_g) < 1e-9,
                    "oracle_hungarian_ms": (t4 - t3) * 1e3, "oracle_same_optimum": abs(s_o - s_g) <= 1e-9 + 1e-13 * abs(s_g)})
    ctx.close()
    last = out[-1]
    print(json.dumps({"metric": "reduced exact solve: host vs GPU path", "unit": "ms",
                      "higher_is_better": False, "data": "synthetic", "results": out,
                      "cpu_baseline": {"value": last["oracle_hungarian_ms"], "unit": "ms", "cores": 1,
                                       "kind": "oracle",
                                       "sample": f"dense O(n^3) Hungarian method of the oracle on the "
                                                 f"n={last['n']} reduced instance (forbidden entries -inf)"}}),
          flush=True)


def run_euclidean(args):
    """The paper's Euclidean random matrix (Sec. 5; n = 1000, 2n points uniform in the unit
    cube, a_ij = exp(-d), quantised to round(2^20 a_ij)) through Algorithm 1 with the
    paper's settings (p = 100, 150, ... on the prescaled scale, eps = t = 1/n, stop at gamma
    <= 2), with the Sinkhorn (step kernel) and the Newton scaling: gamma, final p, O(n^2)
    operations (sweeps / reads of K), remaining entries and time, beside the paper's row
    (Tables 1 and 3: gamma 1.728, p 200, 1416 Sinkhorn iterations / 742 Newton operations,
    0.92 % remaining; a different random instance of the same distribution)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3830_gb300 import api
    from paper_1104_3830_gb300 import workloads as W
    ctx = api.sa_create(0, torch.cuda.current_stream().cuda_stream)
    n = 1000
    w, _, _ = W.euclidean(n, 20261202 + 50)
    d = api.to_device(w)
    out = {}
    with ClockSampler(0) as clk:
        for kernel in ("step", "newton"):
            for _ in range(max(3, args.warmup)):   # warm-up (module load, clocks up)
                api.sa_algorithm1(ctx, d, opt_ratio=2.0, p0=100.0, dp=50.0, max_rounds=30, kernel=kernel,
                                  allow_not_converged=True)
            torch.cuda.synchronize()
            ts = []
            for _ in range(max(3, args.steps)):
                t0 = time.perf_counter()
                g = api.sa_algorithm1(ctx, d, opt_ratio=2.0, p0=100.0, dp=50.0, max_rounds=30, kernel=kernel,
                                      allow_not_converged=True)
                ts.append(time.perf_counter() - t0)
            out[kernel] = {"gamma": g["gamma"], "p_final": g["p_final"], "rounds": g["rounds"],
                           "operations": g["sweeps_total"], "remaining_pct": 100.0 * g["nnz"] / (n * n),
                           "ms": statistics.median(ts) * 1e3, "ms_min": min(ts) * 1e3, "runs": len(ts),
                           "status": g["status"]}
    ctx.close()
    line = {"metric": "Algorithm 1 on the Euclidean random matrix (Tables 1 and 3)", "unit": "ms",
            "higher_is_better": False, "data": "synthetic", "config": {"n": n, "opt_ratio": 2.0,
            "p0": 100.0, "dp": 50.0, "eps": "1/n", "t": "1/n"}, "results": out,
            "paper": {"gamma": 1.728, "p": 200, "sinkhorn_iterations": 1416, "newton_operations": 742,
                      "remaining_pct": 0.92}, "clocks": clk.summary()}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_algorithm1_baseline(w, opt_ratio=2.0, p0=100.0, dp=50.0, max_rounds=30)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="planted8192")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--reduced-sizes", default="1024,2048,4096",
                    help="orders n of the reduced-solve workload, comma-separated")
    ap.add_argument("--kernel", default="auto", choices=["auto", "step", "fused", "plain", "newton"],
                    help="sweep implementation of sa_scale (auto: the library's choice)")
    ap.add_argument("--max-sweeps", type=int, default=20000)
    ap.add_argument("--batch-count", type=int, default=4096)
    ap.add_argument("--plain-sample", type=int, default=64)
    ap.add_argument("--check-sample", type=int, default=32,
                    help="batched form: instances whose certified optimum is compared with the oracle's")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--batch-warmup", type=int, default=1)
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload only: skip the batched and serving parts of the line")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--serve-pool", type=int, default=96)
    ap.add_argument("--serve-dist", default="uniform", choices=["uniform", "zipf"])
    ap.add_argument("--serve-requests", type=int, default=150)
    ap.add_argument("--no-newton", action="store_true",
                    help="skip the Newton-path time-to-solution measurement beside the main line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch4096":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "precision20000":
        return run_precision(args)
    if args.workload == "reduced":
        return run_reduced(args)
    if args.workload == "euclidean1000":
        return run_euclidean(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1104_3830_gb300 import api
    from paper_1104_3830_gb300 import _lib

    w, ps, cfg = workload(args.workload)
    n = w.shape[0]
    stream = torch.cuda.current_stream()
    ctx = api.sa_create(local, stream.cuda_stream)
    d = api.to_device(w, local)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{local}")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        api.sa_assign(ctx, d, ps, 1e-6, args.max_sweeps, kernel=args.kernel)
    barrier()
    times, sweeps, kms, res = [], 0, [], None
    launches0 = _lib.lib().sa_kernel_launches()
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()          # L2 flush between timed steps (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = api.sa_assign(ctx, d, ps, 1e-6, args.max_sweeps, kernel=args.kernel)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            sweeps += res["scale"]["sweeps_total"]
            kms.append(res["scale"]["kernel_ms"])
    launches = (_lib.lib().sa_kernel_launches() - launches0) // args.steps
    barrier()
    total_ms, all_sweeps = over_ranks(sum(times), sweeps, dist, f"cuda:{local}")
    value = all_sweeps / (total_ms / 1e3)

    # roofline of the dominant kernel (the scaling kernel: over 99% of the step).
    # Algorithmic bytes per sweep = n^2 * (bytes per weight): one read of the integer matrix.
    # The step kernel reads its FP32 step matrix instead (n * ceil(n/4)*4 * 4 bytes per
    # sweep), reported beside as bytes_read_per_sweep.
    peak, peak_kind = load_peaks()
    sweeps_per_step = sweeps / args.steps
    kernel_ms = statistics.mean(kms)
    used = res["scale"].get("kernel_used")
    alg_bytes = sweeps_per_step * n * n * w.dtype.itemsize
    achieved = alg_bytes / (kernel_ms / 1e3) / 1e9
    read_per_sweep = (n * ((n + 3) // 4 * 4) * 4) if used in (3, 4) else (n * n * w.dtype.itemsize * (2 if used == 2 else 1))
    traffic, tsrc = measured_traffic(used, n, w.dtype.itemsize)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic * sweeps_per_step if traffic else None,
                "traffic_per_sweep": traffic, "traffic_source": tsrc or "none for this kernel source or size",
                "kernel": KERNEL_NAMES.get(used, "?"),
                "bytes_read_per_sweep": read_per_sweep,
                "frac_of_bytes_read": read_per_sweep * sweeps_per_step / (kernel_ms / 1e3) / 1e9 / peak,
                "peak_source": f"{peak_kind} hbm_gbs", "sweep_us": kernel_ms * 1e3 / max(sweeps_per_step, 1)}

    # end to end through the C ABI with the matrix in pinned host memory
    pinned = torch.from_numpy(np.ascontiguousarray(w)).pin_memory()
    hw = pinned.numpy()
    api.sa_assign_host(ctx, hw, ps, 1e-6, args.max_sweeps, kernel=args.kernel)
    e2e_t, e2e_sw = [], 0
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r2 = api.sa_assign_host(ctx, hw, ps, 1e-6, args.max_sweeps, kernel=args.kernel)
        e1.record(stream)
        e1.synchronize()
        e2e_t.append(e0.elapsed_time(e1))
        e2e_sw += r2["scale"]["sweeps_total"]
    e2e_ms, e2e_all = over_ranks(sum(e2e_t), e2e_sw, dist, f"cuda:{local}")
    e2e_val = e2e_all / (e2e_ms / 1e3)
    d2h = n * 8 + (r2["nnz_final"] + r2["nnz_first"]) * 8 + 8 * (n + 1)
    e2e = {"value": e2e_val, "unit": "sweeps/s", "h2d_bytes_per_step": int(w.nbytes), "d2h_bytes_per_step": int(d2h)}

    # the Newton variant (Sec. 5.3) on the same instance: time to the same certified result
    newton = None
    if not args.no_newton and args.kernel in ("auto", "step"):
        for _ in range(2):
            api.sa_assign(ctx, d, ps, 1e-6, args.max_sweeps, kernel="newton")
        nt_t, nt_reads, rn = [], 0, None
        for _ in range(3):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rn = api.sa_assign(ctx, d, ps, 1e-6, args.max_sweeps, kernel="newton")
            e1.record(stream)
            e1.synchronize()
            nt_t.append(e0.elapsed_time(e1))
            nt_reads += rn["scale"]["sweeps_total"]
        newton = {"kernel": KERNEL_NAMES[4], "ms_per_assign": statistics.mean(nt_t),
                  "reads_of_K_per_assign": nt_reads / 3, "converged": rn["scale"]["converged"],
                  "gamma": rn["gamma"], "ms_scale": rn["ms_scale"],
                  "sinkhorn_ms_per_assign": total_ms / args.steps}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32 (exp/sum), f64 potentials", "data": "synthetic",
                "config": dict(cfg, n=n, sweeps_per_step=sweeps_per_step, parallelism=f"replicas x{world}",
                               l2="flushed between steps (256 MiB write)",
                               impl=KERNEL_NAMES.get(res["scale"].get("kernel_used"), "?"),
                               nnz_first=res["nnz_first"], gamma=res["gamma"], repairs=res["repairs"],
                               ms_scale=res["ms_scale"], ms_prune=res["ms_prune"], ms_solve=res["ms_solve"],
                               ms_certify=res["ms_certify"], converged=res["scale"]["converged"]),
                "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary()}
        if newton is not None:
            line["newton_variant"] = newton
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(w, ps)
    ctx.close()
    if rank == 0:
        # the metric's other two parts, at one GPU (the replicas of a multi-GPU run time
        # only the headline workload)
        if world == 1 and args.workload == "planted8192" and not args.no_extras:
            del d, flush
            torch.cuda.empty_cache()
            line["batched"] = batched_part(args)
            torch.cuda.empty_cache()
            line["serve"] = serve_part(args)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
