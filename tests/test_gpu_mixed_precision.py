"""Mixed precision against the FP64 oracle, result by result, through the C ABI.

Mixed mode keeps K, the iterates, the SpMVs and the Anderson memory in FP32 and
accumulates the Gram matrix, the m x m solve, the safeguard's residual norm and
the KKT norms to FP64 accuracy (float-float pairs per thread and warp, FP64
from there).  These tests state, for each workload, how far the mixed GPU
result is from the FP64 oracle:

* the iterates u^1 .. u^200 against the oracle's FP64 trajectory from the same
  start (relative error ||u_gpu - u_oracle|| / ||u_oracle||, and how many of
  the 200 AA/PDHG decisions differ);
* the primal objective at KKT <= 1e-4 against the exact optimum c'x* of the
  generator (and, on the 200 x 500 LP, against the oracle's own objective at
  1e-4 and at the same iteration count);
* the float-float sums themselves: the Gram matrix and ||g^k|| against FP64
  sums of the very FP32 vectors the device stored.

With AAPDHG_MIXED_RECORD=<path> every measured figure is appended to that file
as one JSON line per result.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
from oracle import oracle as O

pytestmark = pytest.mark.gpu

RECORD = os.environ.get("AAPDHG_MIXED_RECORD")
E32 = float(np.finfo(np.float32).eps)


def _record(name, **kw):
    line = dict(result=name, **kw)
    print(json.dumps(line))
    if RECORD:
        with open(RECORD, "a") as f:
            f.write(json.dumps(line) + "\n")


def _Ksp(P):
    return sp.csr_matrix((P.val, P.col_idx.astype(np.int64), P.row_ptr), shape=(P.m, P.n))


def _rel_obj(a, b):
    return abs(a - b) / (1.0 + abs(b))


def _trajectory(P, solver_setup, prm, iters=200, scaled=False):
    """Relative error of the mixed GPU iterates u^1..u^iters against the FP64
    oracle's, the worst and the last, and the number of differing decisions."""
    from paper_2508_08062_gb300 import Solver
    lp = O.OracleLP.from_problem(P)
    dr = dc = None
    if scaled:
        dr, dc = O.scaling(lp, 10, True)
        lp = O.scaled_lp(lp, dr, dc)
    ref = O.solve(lp, prm, iters, trace=True, rec_len=iters + 1)
    errs = []
    with Solver(P, precision="mixed") as s:
        solver_setup(s)
        s.set_trace(iters)
        s.iterate(0)
        for k in range(iters + 1):
            x, y = s.get_iterate()
            r = ref.rec_u[k]
            if scaled:   # the oracle iterates on the scaled LP: x = Dc x~, y = Dr y~
                r = np.concatenate([dc * r[:P.n], dr * r[P.n:]])
            u = np.concatenate([x, y])
            errs.append(np.linalg.norm(u - r) / np.linalg.norm(r))
            if k < iters:
                s.iterate(1)
        tr = s.get_trace()
    mism = int(np.sum(tr["branch"][:iters] != ref.branch[:iters]))
    return np.array(errs[1:]), mism


def test_tiny_mixed_iterates_and_objective_vs_oracle():
    """200 x 500, AA-PDHG m = 5 (the plain-method workload, here in mixed precision)."""
    P = lpgen.tiny()
    nrm = np.linalg.norm(_Ksp(P).toarray(), 2)
    tau = sig = 0.9 / nrm
    prm = O.Params(method=1, mem=5, tau=tau, sigma=sig)

    def setup(s):
        s.set_steps(tau, sig)
        s.set_method("aa", mem=5)
    errs, mism = _trajectory(P, setup, prm)
    # FP32 data and iterates: a few hundred FP32 ulps early, growing slowly
    assert errs.max() <= 2e-4, errs.max()
    assert mism == 0, mism

    from paper_2508_08062_gb300 import Solver
    lp = O.OracleLP.from_problem(P)
    with Solver(P, precision="mixed") as s:
        setup(s)
        conv, its = s.iterate(200000, tol=1e-4, kkt_every=64)
        x, y = s.get_iterate()
    assert conv
    o_at = O.kkt(lp, x, y)
    assert o_at["kkt"] <= 1.05e-4, o_at
    ref_tol = O.solve(lp, prm, 200000, tol=1e-4, kkt_every=64)
    ref_same = O.solve(lp, prm, its, tol=0.0, kkt_every=0)
    p_gpu = float(P.c @ x)
    p_tol = float(P.c @ ref_tol.x)
    p_same = float(P.c @ ref_same.x)
    vs_star, vs_tol, vs_same = (_rel_obj(p_gpu, P.pobj_star), _rel_obj(p_gpu, p_tol),
                                _rel_obj(p_gpu, p_same))
    _record("tiny 200x500 AA m=5", iterate_err_max=float(errs.max()), iterate_err_200=float(errs[-1]),
            branch_mismatches=mism, gpu_iters=int(its), oracle_iters=int(ref_tol.iters),
            obj_vs_exact=vs_star, obj_vs_oracle_at_1e4=vs_tol, obj_vs_oracle_same_iter=vs_same,
            oracle_kkt_of_gpu_point=o_at["kkt"])
    # The two runs stop at different checks (FP32 moves KKT across 1e-4 a few
    # checks apart), and both points are only 1e-4-optimal, so the objectives
    # differ by ~1e-6 (measured 1.6e-6); at the same iteration count the
    # trajectories have drifted apart by then (measured 1.1e-5).
    assert vs_tol <= 1e-5, vs_tol
    assert vs_same <= 5e-5, vs_same
    assert vs_star <= 1e-4, vs_star


def test_medium_scaled_mixed_iterates_vs_oracle():
    """100k x 300k, Ruiz x10 + Pock-Chambolle, AA-PDHG m = 10: the first 200
    iterates against the oracle's FP64 trajectory on the same scaled LP."""
    P = lpgen.medium()
    from paper_2508_08062_gb300 import Solver
    with Solver(P, precision="mixed") as s:
        s.set_scaling(10, True)
        nrm = s.estimate_norm(100, seed=1)
    tau = sig = 0.9 / nrm
    prm = O.Params(method=1, mem=10, tau=tau, sigma=sig)

    def setup(s):
        s.set_scaling(10, True)
        s.set_steps(tau, sig)
        s.set_method("aa", mem=10)
    errs, mism = _trajectory(P, setup, prm, scaled=True)
    _record("medium 100kx300k scaled AA m=10", iterate_err_max=float(errs.max()),
            iterate_err_200=float(errs[-1]), branch_mismatches=mism)
    assert errs.max() <= 5e-4, errs.max()
    assert mism == 0, mism


def test_medium_scaled_primal_weight_mixed_objective_at_tolerance():
    """The preconditioned 100k x 300k LP with the primal weight update
    (U_P = 3000), mixed, run to KKT <= 1e-4: objective against c'x*, and the
    oracle's KKT of the GPU's point."""
    P = lpgen.medium()
    from paper_2508_08062_gb300 import Solver
    with Solver(P, precision="mixed") as s:
        s.set_scaling(10, True)
        nrm = s.estimate_norm(100, seed=1)
        s.set_steps(0.9 / nrm, 0.9 / nrm)
        s.set_method("aa", mem=10)
        s.set_primal_weight(3000)
        conv, its = s.iterate(200000, tol=1e-4, kkt_every=64)
        x, y = s.get_iterate()
        g = s.get_kkt()
    assert conv
    o = O.kkt(O.OracleLP.from_problem(P), x, y)
    vs_star = _rel_obj(float(P.c @ x), P.pobj_star)
    _record("medium 100kx300k scaled AA m=10 U_P=3000", gpu_iters=int(its), obj_vs_exact=vs_star,
            gpu_kkt=g["kkt"], oracle_kkt_of_gpu_point=o["kkt"])
    assert o["kkt"] <= 1.1e-4, o
    assert vs_star <= 2e-4, vs_star


BATCH_ROWS = (1000, 1500, 2200, 3300, 5000)


def test_batch_members_mixed_vs_oracle():
    """Five members of the batched workload (rows 1k .. 5k, set up as that
    workload: Ruiz x10 + Pock-Chambolle, AA-PDHG m = 10) advanced together in
    mixed precision: each member's first 200 iterates against its own FP64
    oracle trajectory on its scaled LP, then, with the primal weight update
    (U_P = 3000), its objective at KKT <= 1e-4 against c'x*."""
    from paper_2508_08062_gb300 import BatchSolver
    probs = [lpgen.batch_member(lpgen.SEED_BASE * 1000 + 4000 + i, m) for i, m in enumerate(BATCH_ROWS)]
    with BatchSolver(probs, precision="mixed") as b:
        b.set_scaling(10, True)
        nrm = b.estimate_norms(100, seed=1)
    taus = 0.9 / nrm
    scal = []
    refs = []
    for Q, t in zip(probs, taus):
        lp = O.OracleLP.from_problem(Q)
        dr, dc = O.scaling(lp, 10, True)
        scal.append((dr, dc))
        refs.append(O.solve(O.scaled_lp(lp, dr, dc), O.Params(method=1, mem=10, tau=t, sigma=t), 200,
                            trace=True, rec_len=201))
    errs = np.zeros((len(probs), 200))
    branch = np.zeros((len(probs), 200), dtype=np.int64)     # 1: AA step taken at that iteration

    def prepare(b):
        b.set_scaling(10, True)
        b.set_steps(taus, taus)
        b.set_method("aa", mem=10)
    with BatchSolver(probs, precision="mixed") as b:
        prepare(b)
        b.iterate(0)
        aa_prev = b.status()[:, 1].copy()
        for k in range(1, 201):
            b.iterate(1)
            aa_now = b.status()[:, 1]
            branch[:, k - 1] = aa_now - aa_prev
            aa_prev = aa_now.copy()
            for p, ((x, y), rr, (dr, dc), Q) in enumerate(zip(b.get_iterate(), refs, scal, probs)):
                r = rr.rec_u[k]
                r = np.concatenate([dc * r[:Q.n], dr * r[Q.n:]])
                errs[p, k - 1] = np.linalg.norm(np.concatenate([x, y]) - r) / np.linalg.norm(r)
    # a differing safeguard decision (||g^k|| within FP32 rounding of its
    # threshold) starts a different run of the method; up to the first one the
    # trajectories must agree
    first_diff = []
    for p, rr in enumerate(refs):
        d = np.nonzero(branch[p] != (rr.branch[:200] == 1))[0]
        first_diff.append(int(d[0]) + 1 if len(d) else None)
    with BatchSolver(probs, precision="mixed") as b:
        prepare(b)
        b.set_primal_weight(3000)
        b.iterate(200000, tol=1e-4, kkt_every=64)
        sols = b.get_iterate()
        st_tol = b.status()
    for p, (Q, (x, y)) in enumerate(zip(probs, sols)):
        o = O.kkt(O.OracleLP.from_problem(Q), x, y)
        vs_star = _rel_obj(float(Q.c @ x), Q.pobj_star)
        upto = first_diff[p] - 1 if first_diff[p] else 200
        _record(f"batch member {Q.m}x{Q.n} scaled AA m=10",
                iterate_err_max_before_first_differing_decision=float(errs[p, :upto].max()),
                iterate_err_200=float(errs[p, -1]), first_differing_decision=first_diff[p],
                differing_decisions=int(np.sum(branch[p] != (refs[p].branch[:200] == 1))),
                gpu_iters_U_P3000=int(st_tol[p, 0]), converged=bool(st_tol[p, 4]), obj_vs_exact=vs_star,
                oracle_kkt_of_gpu_point=o["kkt"])
    for p, (Q, (x, y)) in enumerate(zip(probs, sols)):
        o = O.kkt(O.OracleLP.from_problem(Q), x, y)
        assert st_tol[p, 4] == 1, p
        assert o["kkt"] <= 1.1e-4, (p, o)
        assert _rel_obj(float(Q.c @ x), Q.pobj_star) <= 2e-4, p
        upto = first_diff[p] - 1 if first_diff[p] else 200
        assert upto >= 50, (p, first_diff[p])
        # measured: 1e-5 .. 1.3e-4 on four members; on the 1500 x 3750 member
        # the FP32 rounding of the data is amplified through a nearly singular
        # Gram system (eta = 1e-10) to 2.4e-2 by iteration 128, where a first
        # decision differs
        assert errs[p, :upto].max() <= 5e-2, (p, errs[p, :upto].max())
    close = [p for p in range(len(probs))
             if errs[p, :(first_diff[p] - 1 if first_diff[p] else 200)].max() <= 5e-4]
    assert len(close) >= 4, close
    assert sum(d is None for d in first_diff) >= 3, first_diff


def test_float_float_gram_and_residual_norm():
    """The Gram matrix, the right-hand side and ||g^k|| that the device
    accumulated in float-float pairs, against FP64 sums of the FP32 vectors the
    device stored (N = 100k elements, AA m = 10, every step accelerated).

    Gram entries and ||g^k||: an FP64 accumulation of the same FP32 terms is
    exact to ~1e-16 per term; a plain FP32 sum would be off by ~1e-5; the
    float-float sums must agree to 1e-12.  The right-hand side <dg_s, g^k>
    is summed directly at every attempt, so it must agree to 1e-12 of
    ||dg_s|| ||g^k|| too."""
    P = lpgen.random_lp(30000, 70000, nnz_per_row=8, frac_ge=0.3, frac_free=0.1, seed=12)
    from paper_2508_08062_gb300 import Solver
    nrm = 0.0
    with Solver(P, precision="mixed") as s:
        nrm = s.estimate_norm(100, seed=1)
        s.set_steps(0.9 / nrm, 0.9 / nrm)
        s.set_method("aa", mem=10, D=1e30)
        s.set_trace(40)
        s.iterate(40)
        mem = s.get_memory()
        tr = s.get_trace()
    k = mem["count"]
    assert k == 10
    dg, g = mem["dg"], mem["g"]
    assert np.all(dg == dg.astype(np.float32)) and np.all(g == g.astype(np.float32))
    G64 = dg @ dg.T
    nrm_cols = np.sqrt(np.diag(G64))
    scale = np.outer(nrm_cols, nrm_cols)
    gram_err = float(np.max(np.abs(mem["gram"] - G64) / scale))
    gn = float(np.linalg.norm(g))
    gn_err = abs(tr["gnorm"][39] - gn) / gn
    rhs64 = dg @ g
    rhs_bound = 1e-12 * nrm_cols * gn
    rhs_err = np.abs(mem["rhs"] - rhs64)
    # what a plain FP32 accumulation of the same Gram entries would give
    G32 = (dg.astype(np.float32) @ dg.T.astype(np.float32)).astype(np.float64)
    gram_err32 = float(np.max(np.abs(G32 - G64) / scale))
    _record("float-float sums, N=100k, m=10", gram_rel_err=gram_err, gnorm_rel_err=gn_err,
            rhs_err_over_bound=float(np.max(rhs_err / rhs_bound)), fp32_gram_rel_err=gram_err32)
    assert gram_err <= 1e-12, gram_err
    assert gn_err <= 1e-12, gn_err
    assert np.all(rhs_err <= rhs_bound), (rhs_err, rhs_bound)
