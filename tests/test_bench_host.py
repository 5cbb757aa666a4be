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


class _FakeLP:
    def __init__(self, m):
        self.m, self.n, self.nnz = m, 2 * m, 8 * m


class _FakeBatch:
    """Stands in for BatchSolver: LP p converges after done_it[p] batch
    iterations (never when done_it[p] is 0)."""
    done_it = None

    def __init__(self, members, precision, stream):
        self.np = len(members)
        self.g = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

    def set_scaling(self, *a): pass
    def set_steps(self, *a): pass
    def set_method(self, *a, **k): pass
    def set_primal_weight(self, **k): pass
    def autotune_layout(self): pass
    def autotune(self): pass

    def estimate_norms(self, *a, **k):
        import numpy as np
        return np.ones(self.np)

    def reset(self):
        self.g = 0

    def iterate(self, n, tol, kkt_every):
        self.g += n
        return bool(all(0 < d <= self.g for d in self.done_it)), n

    def status(self):
        import numpy as np
        st = np.zeros((self.np, 6), dtype=np.int64)
        st[:, 4] = [1 if 0 < d <= self.g else 0 for d in self.done_it]
        return st

    def get_kkt(self):
        import numpy as np
        kk = np.zeros((self.np, 6))
        kk[:, 3] = [1e-4 if 0 < d <= self.g else 3e-3 for d in self.done_it]
        return kk


class _FakeSolver:
    def __init__(self, P, precision, stream):
        self.P = P

    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False

    def set_scaling(self, *a): pass
    def set_steps(self, *a): pass
    def set_method(self, *a, **k): pass
    def set_primal_weight(self, **k): pass

    def estimate_norm(self, *a, **k):
        return 1.0

    def iterate(self, cap, tol, kkt_every):
        return self.P.m != 40, 1000          # the LP with 40 rows does not converge


def test_batched_leg_counts_solved_lps_and_their_latency(monkeypatch):
    """The default line's 256-LP leg with fake solvers: solved LPs, the batch
    iterations until every LP stopped or the cap, per-LP latency percentiles
    over the solved LPs only, and a 4-LP sample of the one-at-a-time solver
    stratified by size."""
    import types
    import lpgen
    import paper_2508_08062_gb300 as pkg
    sizes = [10, 40, 20, 30, 50, 60, 70]
    members = [_FakeLP(m) for m in sizes]
    monkeypatch.setattr(lpgen, "batch", lambda seed: members)
    _FakeBatch.done_it = [64, 128, 0, 64, 192, 320, 0]            # 5 of 7 converge
    monkeypatch.setattr(pkg, "BatchSolver", _FakeBatch, raising=False)
    monkeypatch.setattr(pkg, "Solver", _FakeSolver, raising=False)
    args = types.SimpleNamespace(batch_max_iters=640)
    out = bench.batched_to_tolerance(args, 0, None, lambda: None)
    assert out["nprob"] == 7 and out["solved"] == 5
    assert out["batch_iterations"] == 640                     # two LPs never stop: the cap
    assert out["rows"] == sum(sizes) and out["nnz"] == 8 * sum(sizes)
    t = out["time_to_tol_s"]
    assert t["p50"] is not None and t["p99"] >= t["p50"] >= 0.0
    assert out["solves_per_s"] == out["solved"] / out["wall_s"]
    one = out["single_lp_fp64_one_at_a_time"]
    assert one["sample_rows"] == [10, 30, 50, 70]            # smallest, ..., largest
    assert one["sample_converged"] == 4
    assert out["speedup_vs_single_fp64"] == out["solves_per_s"] / one["solves_per_s"]
    assert out["kkt_max"] == 3e-3
