"""The batched solver at the batched workload's full size (256 LPs, rows
log-uniform in [1k, 50k], cols 2.5x rows, ~8 nnz per row; about 22M nonzeros
in total), in the launch configuration the benchmark times (Ruiz +
Pock-Chambolle scaling, per-problem power-iteration step sizes, AA-PDHG with
m = 10, CUDA-graph chunks of 64 iterations).

What the FP64 oracle can check at this size is checked on sampled members
(the smallest, a median and the largest LP): FP64 iterates of forced AA steps
(every iteration runs the m x m solve and the mix) at 1e-9, and in mixed
precision the KKT quantities of the GPU's iterate re-evaluated by the oracle;
on every member, properties that hold at any size (the iterate lies in X x Y,
the counters add up).
"""
import numpy as np
import pytest

import lpgen
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def members():
    return lpgen.batch()


def _sample(members):
    sizes = np.array([P.m for P in members])
    order = np.argsort(sizes)
    return [int(order[0]), int(order[len(order) // 2]), int(order[-1])]


def test_fullsize_fp64_forced_aa_iterates(members):
    from paper_2508_08062_gb300 import BatchSolver
    iters = 3
    with BatchSolver(members, precision="fp64") as b:
        nrm = b.estimate_norms(30, seed=1)
        tau = 0.9 / nrm
        b.set_steps(tau, tau)
        b.set_method("aa", mem=10, D=1e30)
        b.iterate(0)
        got = [b.get_iterate()]
        for _ in range(iters):
            b.iterate(1)
            got.append(b.get_iterate())
        st = b.status()
    assert np.all(st[:, 0] == iters)
    for p in _sample(members):
        P = members[p]
        ref = O.solve(O.OracleLP.from_problem(P), O.Params(method=1, mem=10, tau=tau[p],
                                                           sigma=tau[p], D=1e30),
                      iters, rec_len=iters + 1)
        assert ref.aa_steps == iters and st[p, 1] == ref.aa_steps
        for k in range(iters + 1):
            u = np.concatenate(got[k][p])
            err = np.linalg.norm(u - ref.rec_u[k]) / np.linalg.norm(ref.rec_u[k])
            assert err <= 1e-9, (p, k, err)


def test_fullsize_mixed_chunk_kkt_and_feasibility(members):
    from paper_2508_08062_gb300 import BatchSolver
    with BatchSolver(members, precision="mixed") as b:
        b.set_scaling(10, True)
        nrm = b.estimate_norms(100, seed=1)
        b.set_steps(0.9 / nrm, 0.9 / nrm)
        b.set_method("aa", mem=10)
        conv, its = b.iterate(128, tol=1e-4, kkt_every=64)
        st = b.status()
        sol = b.get_iterate()
        kk = b.get_kkt()
    assert its == 128
    assert np.all(st[:, 0] + 0 == np.where(st[:, 4] == 1, st[:, 0], 128))
    assert np.all(st[:, 1] + st[:, 2] == st[:, 0]) and np.all(st[:, 5] == 0)
    # x = Dc x~ with x~ clamped to the FP32 bounds of the scaled LP: inside
    # [l, u] up to the rounding of the two products (a few FP32 ulps)
    e = 4 * float(np.finfo(np.float32).eps)
    for p, P in enumerate(members):
        x, y = sol[p]
        assert np.all(x >= P.l - e * np.abs(P.l)) and np.all(x <= P.u + e * np.abs(P.u)), p
        assert np.all(y[P.sense == 1] >= 0), p
    for p in _sample(members):
        o = O.kkt(O.OracleLP.from_problem(members[p]), *sol[p])
        for j, key in enumerate(("r_p", "r_d", "kkt")):
            assert abs(kk[p, j] - o[key]) <= 1e-4 * o[key] + 1e-9, (p, key, kk[p, j], o[key])
