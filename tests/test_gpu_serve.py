"""Served stream (aapdhg_server_*): continuous batching of LPs that arrive
while others are on the GPU.

Every step a member of a cohort takes is computed from that member's data
alone, in the same order as in a batch of one (its rows, its element chunks
and their reductions, its power-iteration segment), and a member joins its
cohort at the cohort's first iteration.  So each LP's result from the server
must equal, bit for bit, the result of the same LP solved alone with the
same set-up; and it must be a 1e-4 (mixed) or 1e-6 (FP64) solution by the
oracle's own KKT evaluation.
"""
import numpy as np
import pytest

import lpgen
from oracle import oracle as O

pytestmark = pytest.mark.gpu


def _alone(P, tol, mem, pw=0):
    from paper_2508_08062_gb300 import BatchSolver
    prec = "fp64" if tol < 1e-5 else "mixed"
    with BatchSolver([P], precision=prec) as b:
        b.set_scaling(10, True)
        nrm = b.estimate_norms(100, seed=1)
        b.set_steps(0.9 / nrm, 0.9 / nrm)
        b.set_method("aa", mem=mem, D=10.0, eps=1.0)
        if pw:
            b.set_primal_weight(period=pw)
        b.set_tolerances([tol])
        conv, _ = b.iterate(200000, tol=tol, kkt_every=64)
        (x, y), = b.get_iterate()
        st = b.status()[0]
    return conv, x, y, int(st[0])


@pytest.mark.parametrize("pw", [0, 500])
def test_server_results_equal_alone_and_meet_their_tolerance(pw):
    # pw > 0: every cohort runs the primal weight update every pw iterations,
    # each LP on its own, so the result alone uses the same setting
    from paper_2508_08062_gb300 import Server
    # (m, n, seed, tol): LPs the oracle takes to their tolerance (scaled as the
    # server scales them) within a few thousand AA iterations; the 1e-6 ones
    # run in FP64 cohorts
    # (with the update every 500 iterations the FP64 oracle itself leaves the
    # 80 x 190 LP of seed 705 above 1e-6 after 200k iterations, so seed 712,
    # which it solves in 8576, takes that place)
    spec = [(60, 150, 700, 1e-4), (120, 300, 701, 1e-6), (90, 200, 702, 1e-4),
            (200, 500, 703, 1e-6), (150, 330, 704, 1e-4), (80, 190, 712 if pw else 705, 1e-6),
            (110, 260, 706, 1e-4)]
    probs = [lpgen.random_lp(m, n, nnz_per_row=5, frac_ge=0.3, frac_free=0.1, seed=sd)
             for m, n, sd, _ in spec]
    tols = [t for *_, t in spec]
    ids, t_sub = [], []
    with Server(method="aa", mem=5, max_cohorts=3, max_cohort_size=2, max_iters=200000) as srv:
        if pw:
            srv.set_primal_weight(period=pw)
        ids.append(srv.submit(probs[0], tols[0]))
        ids.append(srv.submit(probs[1], tols[1]))
        k, rounds, max_running = 2, 0, 0
        while True:
            running, waiting = srv.step()
            max_running = max(max_running, running)
            rounds += 1
            # later LPs arrive one every few rounds, while others are on the GPU
            if k < len(probs) and rounds % 3 == 0:
                ids.append(srv.submit(probs[k], tols[k]))
                k += 1
            if k == len(probs) and running == 0 and waiting == 0:
                break
            assert rounds < 20000
        res = [srv.result(i) for i in ids]
        assert srv.device_bytes() == 0
    assert max_running >= 2                  # cohorts overlapped on the device
    for P, tol, r in zip(probs, tols, res):
        assert r["state"] == "converged", r["state"]
        assert 0 <= r["t_submit"] <= r["t_admit"] <= r["t_done"]
        conv, x, y, its = _alone(P, tol, 5, pw)
        assert conv
        assert r["iters"] == its
        assert np.array_equal(r["x"], x) and np.array_equal(r["y"], y)
        o = O.kkt(O.OracleLP.from_problem(P), r["x"], r["y"])
        # mixed: the GPU's FP32 evaluation may differ from FP64 by a few FP32
        # ulps of the residual's terms near the tolerance
        assert o["kkt"] <= tol * (1.05 if tol >= 1e-5 else 1.0 + 1e-6), (tol, o)


def test_server_hands_back_a_member_before_its_cohort_finishes():
    """Two LPs in one cohort, one needing far more iterations: the fast one's
    result is handed back (state converged, x, y, KKT) by the step that sees it
    converge, while the other still runs, and it equals the LP solved alone."""
    from paper_2508_08062_gb300 import Server
    fast = lpgen.random_lp(60, 150, nnz_per_row=5, frac_ge=0.3, frac_free=0.1, seed=700)
    slow = lpgen.random_lp(1500, 4000, nnz_per_row=8, frac_ge=0.3, frac_free=0.1,
                           row_scale_sigma=1.0, seed=703)
    early = None
    with Server(method="aa", mem=5, max_cohorts=1, max_cohort_size=2, max_iters=20000) as srv:
        a = srv.submit(fast, 1e-4)
        b = srv.submit(slow, 1e-5)
        for _ in range(20000):
            running, waiting = srv.step()
            ra = srv.result(a)
            if early is None and ra["state"] == "converged":
                assert srv.result(b)["state"] == "running" and running == 1
                early = ra
            if running == 0 and waiting == 0:
                break
        final_a, final_b = srv.result(a), srv.result(b)
    assert early is not None
    assert final_b["state"] in ("converged", "capped") and final_b["iters"] > early["iters"]
    assert np.array_equal(early["x"], final_a["x"]) and np.array_equal(early["y"], final_a["y"])
    assert early["iters"] == final_a["iters"] and early["kkt"] == final_a["kkt"]
    conv, x, y, its = _alone(fast, 1e-4, 5)
    assert conv and its == early["iters"]
    assert np.array_equal(early["x"], x) and np.array_equal(early["y"], y)
    assert O.kkt(O.OracleLP.from_problem(fast), x, y)["kkt"] <= 1.05e-4


def test_server_rejects_what_cannot_fit_and_refuses_malformed_input():
    from paper_2508_08062_gb300 import Server
    good = lpgen.random_lp(120, 300, nnz_per_row=5, frac_ge=0.3, frac_free=0.1, seed=701)
    bad = lpgen.random_lp(60, 150, nnz_per_row=5, seed=702)
    bad.col_idx = bad.col_idx.copy()
    bad.col_idx[0] = bad.n                    # column out of range
    with Server(method="aa", mem=5, max_cohorts=2, max_cohort_size=1, max_iters=50000,
                mem_budget=4096) as srv:         # 4 KiB: too small for any LP
        a = srv.submit(good, 1e-4)
        for _ in range(3):
            srv.step()
        assert srv.result(a)["state"] == "rejected"
    from paper_2508_08062_gb300 import AAPDHGError
    with Server(method="aa", mem=5, max_cohorts=2, max_cohort_size=1, max_iters=50000) as srv:
        with pytest.raises(AAPDHGError, match="column index"):
            srv.submit(bad, 1e-4)
        b = srv.submit(good, 1e-4)               # the server goes on
        for _ in range(20000):
            running, waiting = srv.step()
            if running == 0 and waiting == 0:
                break
        assert srv.result(b)["state"] == "converged"


def test_server_primal_weight_rejects_parameters_out_of_range():
    # not sticky: the server goes on with its previous setting
    from paper_2508_08062_gb300 import AAPDHGError, Server
    good = lpgen.random_lp(60, 150, nnz_per_row=5, frac_ge=0.3, frac_free=0.1, seed=700)
    with Server(method="aa", mem=5, max_cohorts=1, max_cohort_size=1, max_iters=200000) as srv:
        with pytest.raises(AAPDHGError, match="primal weight"):
            srv.set_primal_weight(period=-1)
        a = srv.submit(good, 1e-4)
        for _ in range(20000):
            running, waiting = srv.step()
            if running == 0 and waiting == 0:
                break
        assert srv.result(a)["state"] == "converged"
