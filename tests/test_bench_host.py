"""Host logic of bench.py that decides what a JSON line reports (CPU only)."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_committed_traffic_follows_the_kernel_sources():
    tf = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for workload, kinds in (("large", ("xstep", "ystep")), ("batch", ("xstep", "ystep"))):
        for kind in kinds:
            ent = tf[workload][kind]
            key = "batch:" + kind if workload == "batch" else kind
            want = ent["dram_bytes_per_launch"] if ent["kernel_sources"] == bench.kernel_source_hash(key) else None
            assert bench.committed_traffic(workload, kind, 1.0) == want, (workload, kind)
            # a scaled run is not the captured launch
            assert bench.committed_traffic(workload, kind, 0.5) is None
    assert bench.committed_traffic("medium", "ystep", 1.0) is None
    assert bench.committed_traffic("large", "mix", 1.0) is None
    assert bench.committed_traffic("large", "memory", 1.0) is None      # not captured
    assert bench.committed_traffic("batch", "memory", 1.0) is None


def test_traffic_figures_are_close_to_the_algorithmic_bytes():
    # a capture far from the algorithmic bytes (re-reads, a wrong scale factor)
    # would not describe the kernel the bench times
    tf = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    alg = {"large": {"xstep": 545942848, "ystep": 485942848},
           "batch": {"xstep": 379859224, "ystep": 297337464}}
    for workload, kinds in alg.items():
        for kind, a in kinds.items():
            r = tf[workload][kind]["dram_bytes_per_launch"] / a
            assert 0.8 <= r <= 1.1, (workload, kind, r)


def test_rank_reductions():
    assert bench.whole_job_rate(2, 100, 500.0) == 400.0
    assert bench.max_over_ranks(3.5, 1) == 3.5
