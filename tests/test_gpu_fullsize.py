"""Parity at the benchmark's full sizes, through the C ABI.

The medium (100k x 300k, ~2M nnz) and large (2M x 5M, ~50M nnz) workloads are
generated with the benchmark's seeds.  What the FP64 oracle can compute at
these sizes is compared directly:
  - one T step elementwise (mixed precision: within FP32 rounding bounds;
    FP64: 1e-12 relative), from a seeded start;
  - the KKT quantities of the GPU's iterate, re-evaluated by the oracle;
  - FP64 iterates of AA-PDHG: 200 with the experiments' safeguard on the
    medium LP, and a few with the safeguard forced open (every iteration runs
    the m x m solve and the mix at full size);
and properties that hold at any size: the iterate after an AA step is in
X x Y (the projection of Alg. 2), and the counters add up.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
from oracle import oracle as O

pytestmark = pytest.mark.gpu

E32 = np.finfo(np.float32).eps
E64 = np.finfo(np.float64).eps


def _Ksp(P):
    return sp.csr_matrix((P.val, P.col_idx.astype(np.int64), P.row_ptr), shape=(P.m, P.n))


@pytest.fixture(scope="module")
def medium():
    return lpgen.medium(seed=lpgen.SEED_BASE + 2)


@pytest.fixture(scope="module")
def large():
    return lpgen.large(seed=lpgen.SEED_BASE + 3)


def _start(P, seed=11):
    rng = np.random.default_rng(seed)
    lo = np.where(np.isfinite(P.l), P.l, -10.0)
    hi = np.where(np.isfinite(P.u), P.u, 10.0)
    x0 = rng.uniform(lo, hi)
    y0 = rng.standard_normal(P.m)
    y0[P.sense == 1] = np.abs(y0[P.sense == 1])
    return x0, y0


def _steps(s):
    nrm = s.estimate_norm(100, seed=1)
    return 0.9 / nrm, 0.9 / nrm


def _check_T(P, prec, mem):
    from paper_2508_08062_gb300 import Solver
    x0, y0 = _start(P)
    with Solver(P, precision=prec) as s:
        tau, sig = _steps(s)
        s.set_steps(tau, sig)
        s.set_method("aa", mem=mem)
        s.set_start(x0, y0)
        xs, ys = s.get_iterate()
        g = s.get_kkt()
        s.iterate(0)
        x1, y1 = s.get_iterate()
    lp = O.OracleLP.from_problem(P)
    xh, yh = O.T(lp, tau, sig, xs, ys)
    o = O.kkt(lp, xs, ys)
    # forward-error bound of a reordered summation: a few ulps of every
    # magnitude that enters the element (|K|'|y| and |K|(2|xh| + |x|) terms)
    eps = E64 if prec == "fp64" else E32
    Ka = abs(_Ksp(P))
    bx = 16 * eps * (np.abs(xs) + tau * (np.abs(P.c) + Ka.T @ np.abs(ys)))
    by = 16 * eps * (np.abs(ys) + sig * (np.abs(P.q) + Ka @ (2 * np.abs(xh) + np.abs(xs))))
    assert np.all(np.abs(x1 - xh) <= bx + 1e-300)
    assert np.all(np.abs(y1 - yh) <= by + 1e-300)
    rtol = 1e-10 if prec == "fp64" else 1e-4
    for k in ("r_p", "r_d", "kkt", "pobj", "dobj"):
        assert abs(g[k] - o[k]) <= rtol * (abs(o[k]) + 1e-6 * (1 + abs(o["pobj"]))), (k, g[k], o[k])


def test_medium_mixed_T_and_kkt(medium):
    _check_T(medium, "mixed", 10)


def test_medium_fp64_T_and_kkt(medium):
    _check_T(medium, "fp64", 10)


def test_large_mixed_T_and_kkt(large):
    _check_T(large, "mixed", 20)


def test_large_fp64_T_and_kkt(large):
    _check_T(large, "fp64", 20)


def _fp64_trajectory(P, mem, iters, D=1e30):
    from paper_2508_08062_gb300 import Solver
    with Solver(P, precision="fp64") as s:
        tau, sig = _steps(s)
        s.set_steps(tau, sig)
        s.set_method("aa", mem=mem, D=D)
        s.set_trace(iters)
        s.iterate(0)
        got = []
        for k in range(iters + 1):
            x, y = s.get_iterate()
            got.append(np.concatenate([x, y]))
            if k < iters:
                s.iterate(1)
        tr = s.get_trace()
    ref = O.solve(O.OracleLP.from_problem(P),
                  O.Params(method=1, mem=mem, tau=tau, sigma=sig, D=D), iters, trace=True,
                  rec_len=iters + 1)
    for k in range(iters + 1):
        err = np.linalg.norm(got[k] - ref.rec_u[k]) / np.linalg.norm(ref.rec_u[k])
        assert err < 1e-9, (k, err)
    assert np.array_equal(tr["branch"][:iters], ref.branch[:iters])
    return ref


def test_medium_fp64_iterates_paper_parameters(medium):
    # the first 200 iterates with the safeguard of the experiments (D = 10)
    _fp64_trajectory(medium, 10, 200, D=10.0)


def test_medium_fp64_aa_iterates(medium):
    # every step an AA step (safeguard forced open).  With eta = 1e-10 on this
    # badly scaled LP the least-squares solve amplifies rounding differences
    # quickly; the first 20 forced steps stay within 1e-9.
    ref = _fp64_trajectory(medium, 10, 20)
    assert np.all(ref.branch[:20] == 1)


def test_large_fp64_aa_iterates(large):
    # ||K|| is about 4e7 here (lognormal(0,3) row scales): c - K'y cancels terms
    # ~1e7 larger than the iterate, so FP64 summation-order differences alone
    # reach 1.7e-9 of ||u|| at u^4 (measured); u^1..u^3 (two AA steps) are
    # compared at 1e-9, and one step elementwise in test_large_fp64_T_and_kkt
    ref = _fp64_trajectory(large, 20, 2)
    assert np.all(ref.branch[:2] == 1)


def test_large_mixed_aa_steps_feasible_and_kkt(large):
    from paper_2508_08062_gb300 import Solver
    P = large
    with Solver(P, precision="mixed") as s:
        tau, sig = _steps(s)
        s.set_steps(tau, sig)
        s.set_method("aa", mem=20, D=1e30)
        s.iterate(40)
        c = s.counters()
        x, y = s.get_iterate()
        g = s.get_kkt()
    assert c["aa_steps"] + c["pdhg_steps"] == 40 and c["iters"] == 40
    assert c["aa_steps"] >= 30
    # the AA step is followed by the projection onto X x Y (Alg. 2)
    assert np.all(x >= P.l.astype(np.float32)) and np.all(x <= P.u.astype(np.float32))
    assert np.all(y[P.sense == 1] >= 0)
    o = O.kkt(O.OracleLP.from_problem(P), x, y)
    for k in ("r_p", "r_d", "kkt"):
        assert abs(g[k] - o[k]) <= 1e-4 * o[k] + 1e-9, (k, g[k], o[k])
