"""Autotuner of sa_batch_scale's launch plan (which path and launch shape each size bucket of
a batch runs on), by timing the candidates on the GPU at hand.

The batched form scales many independent instances whose sizes spread over [1, 512]: the
smallest run the most sweeps (at high p on uniform weights most n <= 32 instances end at
the sweep cap), so the latency of one sweep decides their time, while the largest are bound
by the SFU work of their elements.  No single launch shape suits both, so instances are
grouped into size buckets and each bucket gets the shape that measured fastest for it:

* the group path (n <= 128): a group of 1, 2 or 4 warps per instance with K in shared
  memory, 1, 2 or 4 groups per block (at most 8 warps per block);
* the register path (n <= 128): K in registers during the sweeps, 1, 2 or 4 warps per
  instance up to n = 32, 4 or 8 up to 64, 16 up to 128 (at most 16 warps per block);
* the K rows path: one block of 256 threads per instance on K kept in a global slot, each
  warp on whole rows;
* the block path: one block of 256 threads per instance, an SFU exp2 per term and sweep.

:func:`tune` times every candidate of every bucket on a seeded synthetic pack of that
bucket (instances/s of sa_batch_scale on that pack alone) and returns the fastest of each;
:func:`load_or_tune` keeps the result in a JSON cache keyed by GPU name, weight type and
bucket, so a later run on the same kind of GPU reuses it.  The plan is applied with
:func:`paper_1104_3830_gb300.api.sa_set_batch_plan`.
"""
from __future__ import annotations

import ctypes
import json
import os
import time

import numpy as np

BUCKETS = [(1, 32), (33, 64), (65, 128), (129, 256), (257, 512)]
GROUP_MAX_N = 128
CACHE_VERSION = 3
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned", "batch_plan.json")


def candidates(lo: int, hi: int):
    """Launch shapes able to run every instance of bucket [lo, hi]: (path, warps per
    instance, groups per block)."""
    if lo < 1 or hi < lo:
        raise ValueError("empty bucket")
    out = []
    if hi <= GROUP_MAX_N:
        out += [("group", w, g) for w in (1, 2, 4) for g in (1, 2, 4) if w * g <= 8]
        regs = (1, 2, 4) if hi <= 32 else (4, 8) if hi <= 64 else (16,)
        out += [("regs", w, g) for w in regs for g in (1, 2, 4, 8) if w * g <= 16]
    out.append(("krows", 0, 0))
    out.append(("block", 0, 0))
    return out


def bucket_name(lo: int, hi: int) -> str:
    return f"{lo}-{hi}"


def plan_from_choice(choice: dict):
    """The sa_set_batch_plan bucket list [(n_hi, path, warps, per_block), ...] for a choice
    {bucket name: (path, warps, per_block)} over BUCKETS (buckets without a choice take the
    block path)."""
    plan = []
    for lo, hi in BUCKETS:
        path, warps, per_block = choice.get(bucket_name(lo, hi), ("block", 0, 0))
        if path in ("group", "regs"):
            if hi > GROUP_MAX_N:
                raise ValueError(f"bucket {lo}-{hi}: the {path} path takes n <= {GROUP_MAX_N}")
            plan.append((hi, path, int(warps), int(per_block)))
        else:
            plan.append((hi, "krows" if path == "krows" else "block", 0, 0))
    return plan


def cache_key(gpu: str, dtype: str) -> str:
    return f"{gpu}|{dtype}"


def load(path: str, gpu: str, dtype: str):
    """The cached choice {bucket: (path, warps, per_block)} for this GPU and weight type, or None (no
    file, another version, no entry, or an entry that is not a valid choice)."""
    try:
        with open(path) as f:
            doc = json.load(f)
    except (OSError, ValueError):
        return None
    if not isinstance(doc, dict) or doc.get("version") != CACHE_VERSION:
        return None
    ent = doc.get("plans", {}).get(cache_key(gpu, dtype))
    if not isinstance(ent, dict):
        return None
    choice = {}
    for lo, hi in BUCKETS:
        b = ent.get(bucket_name(lo, hi))
        if not isinstance(b, dict):
            return None
        c = (b.get("path"), b.get("warps"), b.get("per_block"))
        if c not in candidates(lo, hi):
            return None
        choice[bucket_name(lo, hi)] = c
    return choice


def save(path: str, gpu: str, dtype: str, choice: dict, timings: dict | None = None) -> None:
    """Merge this GPU's and weight type's choice (and the timings behind it) into the cache."""
    try:
        with open(path) as f:
            doc = json.load(f)
        if not isinstance(doc, dict) or doc.get("version") != CACHE_VERSION:
            doc = {}
    except (OSError, ValueError):
        doc = {}
    doc["version"] = CACHE_VERSION
    ent = {}
    for lo, hi in BUCKETS:
        name = bucket_name(lo, hi)
        path_, warps, per_block = choice[name]
        ent[name] = {"path": path_, "warps": int(warps), "per_block": int(per_block)}
        if timings and name in timings:
            ent[name]["instances_per_s"] = {f"{p}:{w}:{g}": v for (p, w, g), v in timings[name].items()}
    doc.setdefault("plans", {})[cache_key(gpu, dtype)] = ent
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(doc, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def bucket_pack(lo: int, hi: int, count: int, dtype, seed: int = 20261202 + 60):
    """A seeded synthetic pack of one bucket: n log-uniform in [lo, hi], weights uniform in
    [1, 1000] (the batched workload's distribution restricted to the bucket)."""
    from . import workloads as W
    ns = W.loguniform_sizes(count, lo, hi, seed + lo)
    return [W.uniform(int(n), 1, 1000, seed, dtype=dtype, tag=7000 + q) for q, n in enumerate(ns)]


class _Pack:
    """A list of host matrices laid out on the device for sa_batch_scale (16-byte rows)."""

    def __init__(self, mats):
        import torch
        esz = mats[0].dtype.itemsize
        ns = np.array([m.shape[0] for m in mats], dtype=np.int32)
        vec = 16 // esz
        lds = ((ns + vec - 1) // vec * vec).astype(np.int64)
        offs = np.concatenate([[0], np.cumsum(lds * ns)[:-1]]).astype(np.int64)
        flat = np.zeros(int((lds * ns).sum()), dtype=mats[0].dtype)
        for m, o, ld in zip(mats, offs, lds):
            n = m.shape[0]
            flat[o:o + n * ld].reshape(n, ld)[:, :n] = m
        self.dev = torch.from_numpy(flat).cuda()
        base = self.dev.data_ptr()
        self.ptrs = torch.tensor([base + esz * int(o) for o in offs], dtype=torch.int64, device="cuda")
        self.n = torch.from_numpy(ns).cuda()
        self.ld = torch.from_numpy(lds).cuda()
        voff = np.concatenate([[0], np.cumsum(ns)[:-1]]).astype(np.int64)
        self.off = torch.from_numpy(voff).cuda()
        tot = int(ns.sum())
        self.u = torch.zeros(tot, dtype=torch.float64, device="cuda")
        self.v = torch.zeros(tot, dtype=torch.float64, device="cuda")
        self.k = len(mats)
        self.wtype = 0 if esz == 2 else 1

    def run(self, ctx, opts):
        from . import _lib as L
        return L.lib().sa_batch_scale(ctx.handle, self.k, ctypes.c_void_p(self.ptrs.data_ptr()),
                                      ctypes.c_void_p(self.n.data_ptr()), ctypes.c_void_p(self.ld.data_ptr()),
                                      ctypes.c_void_p(self.off.data_ptr()), self.wtype, ctypes.byref(opts),
                                      ctypes.c_void_p(self.u.data_ptr()), ctypes.c_void_p(self.v.data_ptr()),
                                      None, None)


def tune(ctx, dtype=np.int32, count_per_bucket: int = 256, ps=None, tol: float = 1e-6, max_sweeps: int = 20000,
         reps: int = 2):
    """Time every candidate of every bucket (instances/s of sa_batch_scale on the bucket's
    pack, best of reps after a warm-up) and return (choice, timings).  The context's plan is
    restored to the library default afterwards."""
    import torch
    from . import _lib as L
    from . import api
    ps = [2.0 ** k for k in range(8)] if ps is None else ps
    opts = L.make_opts(ps, tol, max_sweeps)
    stream = torch.cuda.current_stream()
    choice, timings = {}, {}
    try:
        for lo, hi in BUCKETS:
            name = bucket_name(lo, hi)
            pack = _Pack(bucket_pack(lo, hi, count_per_bucket, dtype))
            timings[name] = {}
            for cand in candidates(lo, hi):
                path, warps, per_block = cand
                # this bucket on the candidate; the pack holds no instance of the others
                plan = [(h, "block", 0, 0) for (_, h) in BUCKETS]
                plan[BUCKETS.index((lo, hi))] = (hi, path, warps, per_block)
                api.sa_set_batch_plan(ctx, plan)
                if pack.run(ctx, opts) == L.SA_E_UNSUPPORTED:   # warm-up; a shape that does not fit
                    continue
                best = float("inf")
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    rc = pack.run(ctx, opts)
                    e1.record(stream)
                    e1.synchronize()
                    if rc not in (L.SA_OK, L.SA_E_NOT_CONVERGED):
                        raise RuntimeError(f"bucket {name}, {cand}: status {rc}: {api.sa_last_error()}")
                    best = min(best, e0.elapsed_time(e1))
                timings[name][cand] = pack.k / (best / 1e3)
            choice[name] = max(timings[name], key=timings[name].get)
    finally:
        api.sa_set_batch_plan(ctx, None)
    return choice, timings


def load_or_tune(ctx, dtype=np.int32, cache: str = DEFAULT_CACHE, **kw):
    """The cached choice for this GPU and weight type, else a fresh one from :func:`tune`
    (saved to the cache).  Returns (plan list for sa_set_batch_plan, choice, source)."""
    import torch
    gpu = torch.cuda.get_device_name()
    dname = np.dtype(dtype).name
    choice = load(cache, gpu, dname)
    if choice is not None:
        return plan_from_choice(choice), choice, f"cache {os.path.basename(cache)}"
    t0 = time.perf_counter()
    choice, timings = tune(ctx, dtype, **kw)
    save(cache, gpu, dname, choice, timings)
    return plan_from_choice(choice), choice, f"tuned now ({time.perf_counter() - t0:.1f} s)"
