"""Host logic of the batched form's autotuner (no GPU): the candidate launch shapes of each
size bucket, the plan built from a choice, and the JSON cache keyed by GPU and weight type."""
import json

import numpy as np
import pytest

from paper_1104_3830_gb300 import autotune as A


def test_candidates_respect_the_group_path_limits():
    for lo, hi in A.BUCKETS:
        c = A.candidates(lo, hi)
        assert ("block", 0, 0) in c and ("krows", 0, 0) in c and len(set(c)) == len(c)
        grp = [x for x in c if x[0] == "group"]
        assert (len(grp) == 8) == (hi <= A.GROUP_MAX_N)
        assert all(w in (1, 2, 4) and g >= 1 and w * g <= 8 for _, w, g in grp)
        regs = [x for x in c if x[0] == "regs"]
        assert bool(regs) == (hi <= A.GROUP_MAX_N)
        # K of a thread's row and column parts fits 64 registers: 2 * n_max / (32 w / n_max) <= 64
        nmax = 32 if hi <= 32 else 64 if hi <= 64 else 128
        assert all(2 * nmax * nmax // (32 * w) <= 64 and w * g <= 16 for _, w, g in regs)
    with pytest.raises(ValueError):
        A.candidates(10, 5)


def test_buckets_cover_the_supported_sizes():
    assert A.BUCKETS[0][0] == 1 and A.BUCKETS[-1][1] == 512
    for (a, b), (c, d) in zip(A.BUCKETS, A.BUCKETS[1:]):
        assert c == b + 1


def test_plan_from_choice():
    choice = {A.bucket_name(lo, hi): (("group", 1, 4) if hi <= 32 else ("block", 0, 0)) for lo, hi in A.BUCKETS}
    plan = A.plan_from_choice(choice)
    assert [h for h, _, _, _ in plan] == [hi for _, hi in A.BUCKETS]
    assert plan[0] == (32, "group", 1, 4) and all(p == "block" and w == 0 for _, p, w, _ in plan[1:])
    with pytest.raises(ValueError):
        A.plan_from_choice({"129-256": ("group", 4, 1)})


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "plan.json")
    assert A.load(path, "GPU A", "int32") is None            # no file yet
    choice = {A.bucket_name(lo, hi): (("group", 2, 4) if hi <= 128 else ("block", 0, 0)) for lo, hi in A.BUCKETS}
    timings = {"1-32": {("group", 2, 4): 1000.0, ("block", 0, 0): 10.0}}
    A.save(path, "GPU A", "int32", choice, timings)
    assert A.load(path, "GPU A", "int32") == choice
    assert A.load(path, "GPU A", "int16") is None            # keyed by weight type
    assert A.load(path, "GPU B", "int32") is None            # and by GPU
    other = dict(choice, **{"1-32": ("group", 1, 1)})
    A.save(path, "GPU B", "int32", other)                    # entries merge
    assert A.load(path, "GPU A", "int32") == choice and A.load(path, "GPU B", "int32") == other
    doc = json.load(open(path))
    assert doc["plans"]["GPU A|int32"]["1-32"]["instances_per_s"]["group:2:4"] == 1000.0
    # a broken entry or another version is not used
    doc["plans"]["GPU A|int32"]["1-32"] = {"path": "group", "warps": 3, "per_block": 1}
    json.dump(doc, open(path, "w"))
    assert A.load(path, "GPU A", "int32") is None
    doc["version"] = A.CACHE_VERSION + 1
    json.dump(doc, open(path, "w"))
    assert A.load(path, "GPU B", "int32") is None
    open(path, "w").write("{not json")
    assert A.load(path, "GPU B", "int32") is None


def test_bucket_pack_is_seeded_and_in_range():
    a = A.bucket_pack(33, 64, 20, np.int16)
    b = A.bucket_pack(33, 64, 20, np.int16)
    assert all(33 <= m.shape[0] <= 64 and m.dtype == np.int16 for m in a)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
