"""GPU (sm_103a) vs FP64 CPU oracle parity, through the C ABI.

FP64 mode: every iterate u^1..u^200 within 1e-9 relative (||du|| / ||u||) and
the same AA / PDHG branch sequence.  Mixed mode (FP32 SpMV and iterates,
FP64-accurate reductions): T and KKT element- and value-wise within bounds
derived from FP32 rounding, and the final objective at KKT <= 1e-4.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
from oracle import oracle as O

pytestmark = pytest.mark.gpu

ITERS = 200
FP64_TOL = 1e-9


def _Ksp(P):
    return sp.csr_matrix((P.val, P.col_idx.astype(np.int64), P.row_ptr), shape=(P.m, P.n))


def _steps(P, safety=0.9):
    from scipy.sparse.linalg import svds
    K = _Ksp(P)
    if P.m == 0 or K.nnz == 0:
        return 1.0, 1.0
    if min(K.shape) <= 2:
        nrm = np.linalg.norm(K.toarray(), 2)
    else:
        nrm = svds(K, k=1, return_singular_vectors=False, random_state=0)[0]
    return safety / nrm, safety / nrm


def _solver(P, prec="fp64"):
    from paper_2508_08062_gb300 import Solver
    return Solver(P, precision=prec)


def _with_long_row_and_column(seed=0, m=300, n=2500):
    """Random LP plus one dense row (n entries: split into chunks) and one
    dense column (m entries), so both matrices exercise every lanes-per-row
    segment and the split-row path."""
    rng = np.random.default_rng(seed)
    base = lpgen.random_lp(m - 1, n, nnz_per_row=6, frac_ge=0.3, frac_free=0.1, seed=seed)
    K = _Ksp(base).tolil()
    K = sp.vstack([K, sp.csr_matrix(rng.standard_normal((1, n)))]).tolil()
    K[:, 7] = rng.standard_normal((m, 1))
    K = K.tocsr()
    K.sort_indices()
    sense = np.concatenate([base.sense, [1]]).astype(np.int8)
    return lpgen.construct(rng, m, n, K.indptr.astype(np.int64), K.indices.astype(np.int32),
                           K.data, sense, base.l, base.u, name="long-row")


def _with_mid_rows(seed=0, m=401, n=3001):
    """Random LP in which 151 rows of K and 41 of its columns hold 33-128
    entries (a few rows a little more): under the default layout they are
    long rows of one chunk each, a warp task per row, next to the SELL slices
    of the short rows."""
    rng = np.random.default_rng(seed)
    base = lpgen.random_lp(m, n, nnz_per_row=5, frac_ge=0.3, frac_free=0.1, seed=seed)
    K = _Ksp(base).tocoo()
    mid_rows = rng.choice(m, 151, replace=False)
    keep = ~np.isin(K.row, mid_rows)
    rows, cols, vals = [K.row[keep]], [K.col[keep]], [K.data[keep]]
    for i in mid_rows:
        c = rng.choice(n, int(rng.integers(33, 129)), replace=False)
        rows.append(np.full(c.size, i)); cols.append(c); vals.append(rng.standard_normal(c.size))
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(m, n)).tocsc()
    mid_cols = rng.choice(n, 41, replace=False)
    A = A.tolil()
    for j in mid_cols:
        r = rng.choice(m, int(rng.integers(33, 100)), replace=False)
        A[r, j] = rng.standard_normal((r.size, 1))
    A = A.tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return lpgen.construct(rng, m, n, A.indptr.astype(np.int64), A.indices.astype(np.int32),
                           A.data, base.sense, base.l, base.u, name="mid-rows")


CASES = {
    "tiny_aa5": (lambda: lpgen.tiny(), dict(method=1, mem=5)),
    "tiny_faa5": (lambda: lpgen.tiny(), dict(method=2, mem=5)),
    "tiny_faa5_literal": (lambda: lpgen.tiny(), dict(method=2, mem=5, faa_adaptive=0)),
    "tiny_pdhg": (lambda: lpgen.tiny(), dict(method=0, mem=0)),
    "mixed_bounds_aa7": (lambda: lpgen.random_lp(333, 777, nnz_per_row=7, frac_ge=0.4,
                                                 frac_free=0.15, frac_lower_only=0.1,
                                                 frac_upper_only=0.1, row_scale_sigma=1.0,
                                                 seed=4),
                         dict(method=1, mem=7, D=1.0, c_div=3.0)),
    "long_rows_aa20": (lambda: _with_long_row_and_column(), dict(method=1, mem=20)),
    "long_rows_faa10": (lambda: _with_long_row_and_column(1), dict(method=2, mem=10)),
    "identity_dhat": (lambda: lpgen.random_lp(50, 90, seed=9), dict(method=1, mem=3,
                                                                    dhat_mode=0, beta=0.5)),
    "mid_rows_aa8": (lambda: _with_mid_rows(), dict(method=1, mem=8)),
    "mid_rows_faa6": (lambda: _with_mid_rows(1), dict(method=2, mem=6)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_fp64_iterates_and_branches_match_oracle(name):
    make, kw = CASES[name]
    P = make()
    tau, sig = _steps(P)
    prm = O.Params(tau=tau, sigma=sig, **kw)
    ref = O.solve(O.OracleLP.from_problem(P), prm, ITERS, trace=True, rec_len=ITERS + 1)
    with _solver(P) as s:
        s.set_steps(tau, sig)
        s.set_method(method=prm.method, mem=prm.mem, D=prm.D, eps=prm.eps, eta=prm.eta,
                     beta=prm.beta, c_s=prm.c_s, kappa=prm.kappa, c_div=prm.c_div,
                     dhat_mode=prm.dhat_mode, faa_adaptive=prm.faa_adaptive)
        s.set_trace(ITERS)
        s.iterate(0)
        worst = 0.0
        for k in range(ITERS + 1):
            x, y = s.get_iterate()
            u = np.concatenate([x, y])
            r = ref.rec_u[k]
            err = np.linalg.norm(u - r) / max(np.linalg.norm(r), 1e-300)
            worst = max(worst, err)
            assert err <= FP64_TOL, (name, k, err)
            if k < ITERS:
                s.iterate(1)
        tr = s.get_trace()
        c = s.counters()
    assert np.array_equal(tr["branch"][:ITERS], ref.branch[:ITERS]), name
    assert np.array_equal(tr["mk"][:ITERS], ref.mk[:ITERS]), name
    assert np.allclose(tr["gnorm"][:ITERS], ref.gnorm[:ITERS], rtol=1e-9, atol=0)
    assert c["aa_steps"] == ref.aa_steps and c["pdhg_steps"] == ref.pdhg_steps
    assert c["iters"] == ITERS


def test_fp64_box_lp_without_constraints():
    # m = 0: K has no rows; x* = l where c > 0, else u (closed form)
    n = 37
    rng = np.random.default_rng(0)
    c = rng.standard_normal(n)
    l = rng.uniform(-5, 0, n)
    u = l + rng.uniform(0.5, 3, n)
    P = lpgen.Problem(0, n, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0),
                      np.zeros(0, np.int8), np.zeros(0), c, l, u)
    with _solver(P) as s:
        s.set_steps(1.0, 1.0)
        s.set_method("aa", mem=3)
        conv, _ = s.iterate(100, tol=1e-14, kkt_every=1)
        x, y = s.get_iterate()
    assert conv and np.array_equal(x, np.where(c > 0, l, u)) and y.size == 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_kkt_at_a_point_matches_oracle(prec):
    P = lpgen.random_lp(400, 900, nnz_per_row=9, frac_ge=0.5, frac_free=0.2,
                        frac_lower_only=0.1, frac_upper_only=0.1, seed=21)
    rng = np.random.default_rng(1)
    x0 = np.clip(P.x_star + 0.1 * rng.standard_normal(P.n), P.l, P.u)
    y0 = P.y_star + 0.1 * rng.standard_normal(P.m)
    y0[P.sense == 1] = np.maximum(y0[P.sense == 1], 0)
    tau, sig = _steps(P)
    with _solver(P, prec) as s:
        s.set_steps(tau, sig)
        s.set_start(x0, y0)
        if prec == "mixed":   # the start is rounded to FP32 on the device
            x0, y0 = s.get_iterate()
        g = s.get_kkt()
    o = O.kkt(O.OracleLP.from_problem(P), x0, y0)
    rtol = 1e-12 if prec == "fp64" else 2e-5
    for k in ("r_p", "r_d", "r_g", "kkt", "pobj", "dobj"):
        assert abs(g[k] - o[k]) <= rtol * (abs(o[k]) + 1e-3 * (1 + abs(o["pobj"]))), (k, g[k], o[k])


def _T_bound(P, x, y, tau, sig, xh):
    """Elementwise FP32 rounding bound of T (mixed mode): a few ulps of every
    magnitude that enters the sum, with the SpMV terms |K||y| and |K||2xh - x|."""
    Ka = abs(_Ksp(P))
    e32 = np.finfo(np.float32).eps
    bx = 16 * e32 * (np.abs(x) + tau * (np.abs(P.c) + Ka.T @ np.abs(y)))
    by = 16 * e32 * (np.abs(y) + sig * (np.abs(P.q) + Ka @ (2 * np.abs(xh) + np.abs(x))))
    return bx, by


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_T_step_elementwise(prec):
    P = _with_long_row_and_column(3)
    rng = np.random.default_rng(2)
    x0 = np.clip(rng.standard_normal(P.n) * 3, P.l, P.u)
    y0 = rng.standard_normal(P.m)
    y0[P.sense == 1] = np.abs(y0[P.sense == 1])
    tau, sig = _steps(P)
    with _solver(P, prec) as s:
        s.set_steps(tau, sig)
        s.set_start(x0, y0)
        xs, ys = s.get_iterate()          # start as stored on the device
        s.iterate(0)                      # u^1 = T u^0
        x1, y1 = s.get_iterate()
    xh, yh = O.T(O.OracleLP.from_problem(P), tau, sig, xs, ys)
    if prec == "fp64":
        assert np.allclose(x1, xh, rtol=1e-13, atol=1e-13)
        assert np.allclose(y1, yh, rtol=1e-13, atol=1e-13)
    else:
        bx, by = _T_bound(P, xs, ys, tau, sig, xh)
        assert np.all(np.abs(x1 - xh) <= bx + 1e-30)
        assert np.all(np.abs(y1 - yh) <= by + 1e-30)


@pytest.mark.parametrize("method", ["aa", "faa"])
def test_mixed_precision_final_objective(method):
    P = lpgen.tiny()
    tau, sig = _steps(P)
    m_id = {"aa": 1, "faa": 2}[method]
    lp = O.OracleLP.from_problem(P)
    ref = O.solve(lp, O.Params(method=m_id, mem=5, tau=tau, sigma=sig), 100000, tol=1e-4,
                  kkt_every=1)
    assert ref.status == 0
    with _solver(P, "mixed") as s:
        s.set_steps(tau, sig)
        s.set_method(method, mem=5)
        conv, its = s.iterate(100000, tol=1e-4, kkt_every=1)
        x, y = s.get_iterate()
        g = s.get_kkt()
    assert conv
    o = O.kkt(lp, x, y)                   # the oracle agrees that the GPU point is converged
    assert o["kkt"] <= 1.05e-4, o
    assert abs(g["kkt"] - o["kkt"]) <= 1e-3 * o["kkt"] + 1e-9
    pref = float(P.c @ ref.x)
    # both points are 1e-4-optimal and stop at different checks; measured
    # objective differences are ~1e-6 (tests/test_gpu_mixed_precision.py states them)
    assert abs(o["pobj"] - pref) <= 2e-5 * (1 + abs(pref)), (o["pobj"], pref)
    print(method, "gpu iters", its, "oracle iters", ref.iters, "rel obj diff",
          abs(o["pobj"] - pref) / (1 + abs(pref)))


def test_resume_and_tolerance_semantics():
    P = lpgen.tiny()
    tau, sig = _steps(P)
    with _solver(P, "fp64") as s:
        s.set_steps(tau, sig)
        s.set_method("aa", mem=5)
        conv1, it1 = s.iterate(150)
        conv2, it2 = s.iterate(150)
        x, y = s.get_iterate()
        assert not conv1 and not conv2 and it1 == 150 and it2 == 150
        ref = O.solve(O.OracleLP.from_problem(P), O.Params(method=1, mem=5, tau=tau, sigma=sig),
                      300)
        assert np.linalg.norm(np.concatenate([x - ref.x, y - ref.y])) <= \
            FP64_TOL * np.linalg.norm(np.concatenate([ref.x, ref.y]))
        conv, its = s.iterate(100000, tol=1e-4, kkt_every=1)
        assert conv
        again, its2 = s.iterate(10, tol=1e-4, kkt_every=1)   # already converged: no work
        assert again and its2 == 0
        assert s.get_kkt()["kkt"] <= 1e-4


def test_invalid_inputs_rejected():
    from paper_2508_08062_gb300 import AAPDHGError
    P = lpgen.random_lp(10, 20, seed=0)
    bad = lpgen.random_lp(10, 20, seed=0)
    bad.col_idx = bad.col_idx.copy()
    bad.col_idx[0] = 20                      # column out of range
    with pytest.raises(AAPDHGError):
        _solver(bad)
    bad = lpgen.random_lp(10, 20, seed=0)
    bad.l = bad.l.copy(); bad.l[3] = bad.u[3] + 1   # l > u
    with pytest.raises(AAPDHGError):
        _solver(bad)
    with _solver(P) as s:
        with pytest.raises(AAPDHGError):
            s.iterate(1)                     # no step sizes yet
    with _solver(P) as s:
        with pytest.raises(AAPDHGError):
            s.set_method("aa", mem=33)


# --------------------------------------------------------------------------
# Diagonal preconditioning (Ruiz x10 + Pock-Chambolle, the Sec. 5.2 set-up)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("method", [1, 2])
def test_fp64_scaled_iterates_match_oracle(method):
    P = lpgen.random_lp(300, 650, nnz_per_row=6, frac_ge=0.4, frac_free=0.15, frac_lower_only=0.1,
                        frac_upper_only=0.1, row_scale_sigma=2.0, seed=17)
    lp = O.OracleLP.from_problem(P)
    dr, dc = O.scaling(lp, 10, True)
    S = O.scaled_lp(lp, dr, dc)
    from scipy.sparse.linalg import svds
    Ks = sp.csr_matrix((S.v, S.ci.astype(np.int64), S.rp), shape=(P.m, P.n))
    tau = sig = 0.9 / svds(Ks, k=1, return_singular_vectors=False, random_state=0)[0]
    prm = O.Params(method=method, mem=6, tau=tau, sigma=sig)
    ref = O.solve(S, prm, ITERS, trace=True, rec_len=ITERS + 1)
    with _solver(P) as s:
        s.set_scaling(10, True)
        s.set_steps(tau, sig)
        s.set_method(method=method, mem=6)
        s.set_trace(ITERS)
        s.iterate(0)
        for k in range(ITERS + 1):
            x, y = s.get_iterate()
            r = np.concatenate([dc * ref.rec_u[k][:P.n], dr * ref.rec_u[k][P.n:]])
            err = np.linalg.norm(np.concatenate([x, y]) - r) / np.linalg.norm(r)
            assert err <= FP64_TOL, (k, err)
            if k < ITERS:
                s.iterate(1)
        tr = s.get_trace()
        g = s.get_kkt()
    assert np.array_equal(tr["branch"][:ITERS], ref.branch[:ITERS])
    o = O.kkt(lp, x, y)                       # KKT in the caller's (unscaled) units
    for k in ("r_p", "r_d", "r_g", "kkt", "pobj", "dobj"):
        assert abs(g[k] - o[k]) <= 1e-10 * (abs(o[k]) + 1e-6), (k, g[k], o[k])


def test_scaling_only_once_and_start_in_caller_units():
    from paper_2508_08062_gb300 import AAPDHGError
    P = lpgen.random_lp(50, 80, row_scale_sigma=2.0, seed=2)
    rng = np.random.default_rng(0)
    x0 = np.clip(rng.standard_normal(P.n), P.l, P.u)
    y0 = np.abs(rng.standard_normal(P.m))
    with _solver(P) as s:
        s.set_scaling(10, True)
        s.set_steps(0.1, 0.1)
        s.set_start(x0, y0)
        x, y = s.get_iterate()
        assert np.allclose(x, x0, rtol=1e-14) and np.allclose(y, y0, rtol=1e-14)
        with pytest.raises(AAPDHGError):
            s.set_scaling(10, True)


# --------------------------------------------------------------------------
# Autotuning of the half-step task shapes: the shape never changes a result
# --------------------------------------------------------------------------
@pytest.mark.parametrize("lp", ["long_row_and_column", "mid_rows"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_task_shapes_give_identical_iterates(prec, lp):
    P = _with_long_row_and_column(3) if lp == "long_row_and_column" else _with_mid_rows(3)
    tau, sig = _steps(P)
    got = []
    for shapes in ((0, 0), (1, 1), (2, 2), (3, 4), (4, 3), None):
        with _solver(P, prec) as s:
            s.set_steps(tau, sig)
            s.set_method("aa", mem=8, D=1e30)
            if shapes is None:
                t = s.autotune()
                assert t["shape_x"] in range(5) and t["shape_y"] in range(5)
                assert all(v > 0 for v in t["x_us"] + t["y_us"])
            else:
                s.set_task_shape(*shapes)
            s.iterate(40)
            x, y = s.get_iterate()
            got.append(np.concatenate([x, y]))
    # rows are summed in the same order under every shape; only the block
    # partials of ||g|| differ in order (they decide nothing with D = 1e30)
    for u in got[1:]:
        assert np.array_equal(u, got[0])
    with _solver(P, prec) as s:
        from paper_2508_08062_gb300 import AAPDHGError
        with pytest.raises(AAPDHGError):
            s.set_task_shape(5, 0)


@pytest.mark.parametrize("layout", [(16, 1024), (64, 512), (128, 2048), (1, 32), (64, 4096, 16, 64)])
def test_fp64_iterates_match_oracle_under_other_layouts(layout):
    """Rows move between the SELL slices (one lane per row) and the long-row
    chunks (a warp per chunk) with the slice width limit, and long rows split
    at other points with the chunk length: the sums run in another order, so
    the FP64 iterates must still follow the oracle within 1e-9, with the same
    branches.  (1, 32): every row but the empty ones is a long row, in
    one-warp chunks of 32 entries.  (64, 4096, 16, 64): K' and K in different
    layouts."""
    P = _with_long_row_and_column(5)
    tau, sig = _steps(P)
    prm = O.Params(tau=tau, sigma=sig, method=1, mem=8)
    ref = O.solve(O.OracleLP.from_problem(P), prm, ITERS, trace=True, rec_len=ITERS + 1)
    with _solver(P) as s:
        s.set_layout(*layout)
        s.set_steps(tau, sig)
        s.set_method("aa", mem=8)
        s.set_trace(ITERS)
        s.iterate(0)
        for k in range(ITERS + 1):
            x, y = s.get_iterate()
            r = ref.rec_u[k]
            err = np.linalg.norm(np.concatenate([x, y]) - r) / np.linalg.norm(r)
            assert err <= FP64_TOL, (layout, k, err)
            if k < ITERS:
                s.iterate(1)
        tr = s.get_trace()
    assert np.array_equal(tr["branch"][:ITERS], ref.branch[:ITERS])


def test_layout_autotuner_keeps_a_candidate_and_the_results():
    P = _with_long_row_and_column(6)
    tau, sig = _steps(P)
    with _solver(P, "mixed") as s:
        s.set_steps(tau, sig)
        s.set_method("aa", mem=5)
        s.iterate(30)
        x0, y0 = s.get_iterate()
        t = s.autotune_layout()                 # the run state is kept
        assert t["x"] in s.LAYOUT_CANDIDATES and t["y"] in s.LAYOUT_CANDIDATES
        bx = min(c["x_us"] for c in t["candidates"])
        by = min(c["y_us"] for c in t["candidates"])
        assert [c["x_us"] for c in t["candidates"] if (c["sell_max"], c["long_chunk"]) == t["x"]][0] == bx
        assert [c["y_us"] for c in t["candidates"] if (c["sell_max"], c["long_chunk"]) == t["y"]][0] == by
        assert all(c["x_us"] > 0 and c["y_us"] > 0 for c in t["candidates"])
        x1, y1 = s.get_iterate()
        assert np.array_equal(x0, x1) and np.array_equal(y0, y1)
        k0 = s.get_kkt()["kkt"]
        s.iterate(3000)                         # the run goes on under the chosen layout
        assert s.counters()["iters"] == 3030
        assert np.isfinite(s.get_kkt()["kkt"]) and s.get_kkt()["kkt"] < k0
        from paper_2508_08062_gb300 import AAPDHGError
        with pytest.raises(AAPDHGError):
            s.set_layout(32, 100)               # not a multiple of 32


# --------------------------------------------------------------------------
# Primal weight update with memory reset and D-hat re-blend (readings R13-R15)
# --------------------------------------------------------------------------
PW_CASES = {
    "aa5_pw": dict(method=1, mem=5),
    "faa5_pw": dict(method=2, mem=5),
    "pdhg_pw": dict(method=0, mem=0),
    "aa5_pw_theta1_noblend": dict(method=1, mem=5, pw_theta=1.0, pw_dhat=0),
}


@pytest.mark.parametrize("name", list(PW_CASES))
def test_fp64_primal_weight_iterates_match_oracle(name):
    P = lpgen.random_lp(333, 777, nnz_per_row=7, frac_ge=0.4, frac_free=0.15, frac_lower_only=0.1,
                        frac_upper_only=0.1, row_scale_sigma=1.0, seed=4)
    tau, sig = _steps(P)
    sig *= 4.0                                     # omega^0 = 2: the steps differ from the start
    tau /= 4.0
    kw = dict(PW_CASES[name])
    prm = O.Params(tau=tau, sigma=sig, pw_period=50, **kw)
    ref = O.solve(O.OracleLP.from_problem(P), prm, ITERS, trace=True, rec_len=ITERS + 1)
    with _solver(P) as s:
        s.set_steps(tau, sig)
        s.set_method(method=prm.method, mem=prm.mem)
        s.set_primal_weight(period=50, theta=prm.pw_theta, eps_zero=prm.pw_eps_zero,
                            dhat_blend=bool(prm.pw_dhat), rho_min=prm.pw_rho_min)
        s.set_trace(ITERS)
        s.iterate(0)
        for k in range(ITERS + 1):
            x, y = s.get_iterate()
            u = np.concatenate([x, y])
            err = np.linalg.norm(u - ref.rec_u[k]) / np.linalg.norm(ref.rec_u[k])
            assert err <= FP64_TOL, (name, k, err)
            if k < ITERS:
                s.iterate(1)
        tr = s.get_trace()
    assert np.array_equal(tr["branch"][:ITERS], ref.branch[:ITERS]), name
    # the update iterations are plain steps
    assert all(tr["branch"][k - 1] == 0 for k in (50, 100, 150))


def test_mixed_primal_weight_stays_bounded_at_fp32_accuracy():
    # a member of the 256-LP batched workload: in mixed precision its KKT
    # stalls near 1e-4 (FP32's attainable accuracy for it); an update driven
    # by the rounding noise of Delta_x, Delta_y there made omega drift and
    # the run diverge (KKT 1e11 after 100k iterations).  With FP32 iterates an
    # update is applied only while the KKT still improves, and the run
    # reaches 1e-4 (about 43k iterations); FP64 needs no such rule (31k).
    ms = lpgen.batch_sizes()
    P = lpgen.batch_member((lpgen.SEED_BASE + 4) * 1000 + 135, int(ms[135]))
    with _solver(P, "mixed") as s:
        s.set_scaling(10, True)
        nrm = s.estimate_norm(100, seed=1)
        s.set_steps(0.9 / nrm, 0.9 / nrm)
        s.set_method("aa", mem=10, D=10.0, eps=1.0)
        s.set_primal_weight(period=3000)
        conv, its = s.iterate(100000, tol=1e-4, kkt_every=64)
        x, y = s.get_iterate()
    assert conv, its
    assert O.kkt(O.OracleLP.from_problem(P), x, y)["kkt"] <= 1.05e-4


def test_mixed_primal_weight_converges():
    P = lpgen.tiny()
    tau, sig = _steps(P)
    with _solver(P, "mixed") as s:
        s.set_steps(tau, sig)
        s.set_method("aa", mem=5)
        s.set_primal_weight(period=500)
        conv, its = s.iterate(100000, tol=1e-4, kkt_every=64)
        x, y = s.get_iterate()
    assert conv
    assert O.kkt(O.OracleLP.from_problem(P), x, y)["kkt"] <= 1.05e-4


@pytest.mark.parametrize("prec,method", [("fp64", "aa"), ("mixed", "aa"), ("mixed", "faa")])
def test_graph_chunks_equal_single_launches(prec, method):
    """Full chunks of 64 iterations run as CUDA graphs; single iterations
    launch every kernel directly.  Both must give the same iterates and
    counters bit for bit, with AA steps both taken and refused along the way."""
    P = lpgen.random_lp(400, 1000, nnz_per_row=6, frac_ge=0.3, frac_free=0.1, seed=17)
    tau, sig = _steps(P)
    res = []
    for chunked in (True, False):
        with _solver(P, prec) as s:
            s.set_steps(tau, sig)
            s.set_method(method, mem=6, D=10.0, eps=1.0)
            s.set_task_shape(1, 1)        # the same grids: ||g|| summed in the same order
            if chunked:
                s.iterate(640, tol=0.0, kkt_every=64)
            else:
                for _ in range(640):
                    s.iterate(1, tol=0.0, kkt_every=64)
            x, y = s.get_iterate()
            res.append((np.concatenate([x, y]), s.counters()))
    (u1, c1), (u2, c2) = res
    assert 0 < c1["aa_steps"] < 640, c1
    assert c1 == c2
    assert np.array_equal(u1, u2)
