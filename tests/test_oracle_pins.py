"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks a closed form,
an invariant, a brute-force answer on a tiny input, a library routine, or a
value the paper prints.  A plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand) fails at least one of them.
"""
import itertools
import json
import os

import numpy as np
import pytest

import lpgen
from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _norm_K(P):
    import scipy.sparse as sp
    K = sp.csr_matrix((P.val, P.col_idx.astype(np.int64), P.row_ptr), shape=(P.m, P.n)).toarray()
    return np.linalg.norm(K, 2) if K.size else 0.0, K


def _steps(P, safety=0.9):
    nrm, _ = _norm_K(P)
    s = safety / nrm
    return s, s


# --------------------------------------------------------------------------
# The toy feasibility LP of Sec. 5.2 (golden: the paper prints the optimum
# (3, 0) and the step 0.1)
# --------------------------------------------------------------------------
def _toy():
    g = json.load(open(os.path.join(GOLDEN, "toy_feasibility.json")))
    P = lpgen.from_dense(g["K"], g["sense"], g["q"], g["c"], g["l"],
                         [float(v) for v in g["u"]], name="toy")
    return g, P


def test_toy_fixed_point_and_convergence():
    g, P = _toy()
    lp = O.OracleLP.from_problem(P)
    x_opt, y_opt = g["optimum_xy"]
    xh, yh = O.T(lp, g["step"], g["step"], [x_opt], [y_opt])
    assert xh[0] == x_opt and yh[0] == y_opt
    for method in (0, 1):
        prm = O.Params(method=method, mem=g["aa_memory"], tau=g["step"], sigma=g["step"],
                       D=1e6, dhat_mode=0)
        r = O.solve(lp, prm, 20000, tol=1e-12, kkt_every=1)
        assert r.status == 0
        assert abs(r.x[0] - x_opt) < 1e-9 and abs(r.y[0] - y_opt) < 1e-9


def test_toy_aa_faster_than_pdhg():
    # Sec. 5.2 reports that AA-PDHG reaches (3, 0) in a few iterations while
    # PDHG spirals; check only the ordering, not a count.
    g, P = _toy()
    lp = O.OracleLP.from_problem(P)
    its = {}
    for method in (0, 1):
        prm = O.Params(method=method, mem=5, tau=0.1, sigma=0.1, D=1e6, dhat_mode=0)
        its[method] = O.solve(lp, prm, 20000, tol=1e-8, kkt_every=1).iters
    assert its[1] < its[0] / 5


# --------------------------------------------------------------------------
# T fixes the constructed optimum (Fix T = KKT points, Sec. 3.1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_T_fixes_constructed_optimum(seed):
    P = lpgen.random_lp(40, 70, nnz_per_row=6, frac_ge=0.4, frac_free=0.2, frac_lower_only=0.15,
                        frac_upper_only=0.15, seed=seed)
    lp = O.OracleLP.from_problem(P)
    tau, sig = _steps(P)
    xh, yh = O.T(lp, tau, sig, P.x_star, P.y_star)
    assert np.max(np.abs(xh - P.x_star)) <= 1e-12 * (1 + np.max(np.abs(P.x_star)))
    assert np.max(np.abs(yh - P.y_star)) <= 1e-12 * (1 + np.max(np.abs(P.y_star)))


def test_T_moves_a_non_optimal_point():
    P = lpgen.random_lp(30, 50, seed=3)
    lp = O.OracleLP.from_problem(P)
    tau, sig = _steps(P)
    xh, yh = O.T(lp, tau, sig, P.x_star + 0.1, P.y_star)
    assert np.max(np.abs(xh - (P.x_star + 0.1))) > 1e-3 or np.max(np.abs(yh - P.y_star)) > 1e-3


def test_T_closed_form_diagonal_lp():
    # min c'x s.t. diag(d) x = q, x free: x* = q/d, y* = c/d (powers of two: exact)
    d = np.array([2.0, 4.0, 0.5, 1.0])
    q = np.array([1.0, -2.0, 3.0, 0.25])
    c = np.array([0.5, 1.0, -1.5, 2.0])
    P = lpgen.from_dense(np.diag(d), np.zeros(4), q, c, np.full(4, -np.inf), np.full(4, np.inf))
    lp = O.OracleLP.from_problem(P)
    xs, ys = q / d, c / d
    xh, yh = O.T(lp, 0.125, 0.25, xs, ys)
    assert np.array_equal(xh, xs) and np.array_equal(yh, ys)
    # one step from the origin, by hand: xh = tau*(K'y - c) = -tau c; yh = sigma (q - K(2xh))
    xh, yh = O.T(lp, 0.125, 0.25, np.zeros(4), np.zeros(4))
    assert np.array_equal(xh, -0.125 * c)
    assert np.array_equal(yh, 0.25 * (q - d * (2 * (-0.125 * c))))
    k = O.kkt(lp, xs, ys)
    assert k["kkt"] == 0.0


def test_T_box_lp_closed_form():
    # K = 0 (one all-zero '=' row with q = 0): optimum x_j = l_j if c_j > 0, else u_j
    n = 6
    c = np.array([1.0, -2.0, 0.5, -0.25, 3.0, -1.0])
    l = np.array([0.0, -1.0, 2.0, -3.0, 0.5, 1.0])
    u = l + np.array([1.0, 2.0, 3.0, 4.0, 5.0, 6.0])
    P = lpgen.Problem(1, n, np.array([0, 0], np.int64), np.zeros(0, np.int32), np.zeros(0),
                      np.zeros(1, np.int8), np.zeros(1), c, l, u)
    lp = O.OracleLP.from_problem(P)
    r = O.solve(lp, O.Params(method=0, mem=0, tau=1.0, sigma=1.0), 200, tol=1e-14,
                kkt_every=1)
    x_star = np.where(c > 0, l, u)
    assert r.status == 0 and np.array_equal(r.x, x_star)


# --------------------------------------------------------------------------
# KKT (Remark on termination conditions; Lambda of eq. lambda-case)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 5])
def test_kkt_zero_at_optimum_positive_off_it(seed):
    P = lpgen.random_lp(50, 90, frac_ge=0.5, frac_free=0.2, frac_lower_only=0.1,
                        frac_upper_only=0.1, seed=seed)
    lp = O.OracleLP.from_problem(P)
    k = O.kkt(lp, P.x_star, P.y_star)
    assert k["kkt"] < 1e-13
    assert abs(k["pobj"] - P.c @ P.x_star) < 1e-12 * (1 + abs(k["pobj"]))
    k2 = O.kkt(lp, P.x_star, P.y_star + 0.01)
    assert k2["r_d"] > 1e-6
    k3 = O.kkt(lp, P.x_star + 0.01, P.y_star)
    assert k3["r_p"] > 1e-6


def _one_var(c, l, u, K=1.0, q=0.0, sense=0):
    return O.OracleLP.from_problem(lpgen.from_dense([[K]], [sense], [q], [c], [l], [u]))


def test_kkt_lambda_cases():
    # c - K'y = 2 - y.  With y = 1: residual r = 1 (positive), y = 3: r = -1.
    # free: Lambda = {0}, lambda = 0, r_d = |r| / (1 + |c|)
    assert O.kkt(_one_var(2.0, -np.inf, np.inf), [0.0], [1.0])["r_d"] == pytest.approx(1 / 3)
    assert O.kkt(_one_var(2.0, -np.inf, np.inf), [0.0], [3.0])["r_d"] == pytest.approx(1 / 3)
    # lower bound only: Lambda = R+, positive r absorbed, negative r not
    assert O.kkt(_one_var(2.0, 0.0, np.inf), [0.0], [1.0])["r_d"] == 0.0
    assert O.kkt(_one_var(2.0, 0.0, np.inf), [0.0], [3.0])["r_d"] == pytest.approx(1 / 3)
    # upper bound only: Lambda = R-
    assert O.kkt(_one_var(2.0, -np.inf, 5.0), [0.0], [1.0])["r_d"] == pytest.approx(1 / 3)
    assert O.kkt(_one_var(2.0, -np.inf, 5.0), [0.0], [3.0])["r_d"] == 0.0
    # boxed: Lambda = R, always absorbed
    assert O.kkt(_one_var(2.0, 0.0, 5.0), [0.0], [3.0])["r_d"] == 0.0


def test_kkt_dual_objective_and_gap_by_hand():
    # min 2x s.t. x = 1 ('='), 0 <= x <= 5.  At x = 1, y = 1.5: c - K'y = 0.5 = lambda
    # (boxed -> lambda = 0.5 = lambda+), dobj = q y + l lambda+ - u lambda- = 1.5 + 0 = 1.5
    lp = _one_var(2.0, 0.0, 5.0, q=1.0)
    k = O.kkt(lp, [1.0], [1.5])
    assert k["pobj"] == 2.0 and k["dobj"] == 1.5
    assert k["r_g"] == pytest.approx(0.5 / (1 + 1.5 + 2.0))
    # same with y = 3: lambda = -1 = -lambda-, dobj = 3 - 5 * 1 = -2
    k = O.kkt(lp, [1.0], [3.0])
    assert k["dobj"] == -2.0
    # lower bound 0.5 and lambda+ = 0.5: dobj = 1.5 + 0.5 * 0.5
    lp = _one_var(2.0, 0.5, 5.0, q=1.0)
    assert O.kkt(lp, [1.0], [1.5])["dobj"] == 1.75


def test_kkt_primal_residual_senses():
    # '>=' row: only a violation counts; '=' row: both signs count
    ge = _one_var(0.0, -np.inf, np.inf, q=1.0, sense=1)
    assert O.kkt(ge, [2.0], [0.0])["r_p"] == 0.0
    assert O.kkt(ge, [0.0], [0.0])["r_p"] == pytest.approx(1.0 / 2.0)
    eq = _one_var(0.0, -np.inf, np.inf, q=1.0, sense=0)
    assert O.kkt(eq, [2.0], [0.0])["r_p"] == pytest.approx(1.0 / 2.0)
    assert O.kkt(eq, [0.0], [0.0])["r_p"] == pytest.approx(1.0 / 2.0)


# --------------------------------------------------------------------------
# D-hat (Remark on its construction), hand-worked
# --------------------------------------------------------------------------
def test_dhat_by_hand():
    # K = [[1, -4, 0, 0], [0, 0.25, 9, 0]]: column maxima 1, 4, 9, 0 -> sqrt -> 1, 2, 3, 1e-5
    # row maxima 4, 9 -> 2, 3
    K = [[1.0, -4.0, 0.0, 0.0], [0.0, 0.25, 9.0, 0.0]]
    P = lpgen.from_dense(K, [0, 1], [0, 0], [0] * 4, [0] * 4, [1] * 4)
    dx, dy = O.dhat(O.OracleLP.from_problem(P), 1)
    assert np.allclose(dx, [1.0, 2.0, 3.0, 1e-5], rtol=1e-15, atol=0)
    assert np.allclose(dy, [2.0, 3.0], rtol=1e-15, atol=0)
    dx, dy = O.dhat(O.OracleLP.from_problem(P), 0)
    assert np.all(dx == 1) and np.all(dy == 1)


# --------------------------------------------------------------------------
# M-Fejer decrease of plain PDHG: ||u+ - u*||_M^2 <= ||u - u*||_M^2 - ||u+ - u||_M^2
# with the symmetric metric M = [[I/tau, K'], [K, I/sigma]] (the firm
# non-expansiveness behind eq. kpd_PDHG-used-1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1])
def test_pdhg_M_fejer(seed):
    P = lpgen.random_lp(30, 45, frac_ge=0.5, frac_free=0.2, frac_lower_only=0.1,
                        frac_upper_only=0.1, seed=seed)
    lp = O.OracleLP.from_problem(P)
    tau, sig = _steps(P, 0.7)
    _, K = _norm_K(P)
    n, m = P.n, P.m
    M = np.block([[np.eye(n) / tau, K.T], [K, np.eye(m) / sig]])
    us = np.concatenate([P.x_star, P.y_star])
    r = O.solve(lp, O.Params(method=0, mem=0, tau=tau, sigma=sig), 300, rec_len=301)
    U = r.rec_u
    for k in range(len(U) - 1):
        a, b = U[k] - us, U[k + 1] - us
        d = U[k + 1] - U[k]
        assert b @ M @ b <= a @ M @ a - d @ M @ d + 1e-9 * (1 + a @ M @ a)


# --------------------------------------------------------------------------
# Whole solver against brute force (vertex enumeration) and HiGHS
# --------------------------------------------------------------------------
def _vertex_enum(P, K):
    """min c'x over the polytope by enumerating basic feasible solutions."""
    n = P.n
    cons = []  # (row, rhs, kind) kind: 'eq', 'ge'
    for i in range(P.m):
        cons.append((K[i], P.q[i], "eq" if P.sense[i] == 0 else "ge"))
    for j in range(n):
        e = np.zeros(n); e[j] = 1.0
        cons.append((e, P.l[j], "ge"))
        cons.append((-e, -P.u[j], "ge"))
    eqs = [i for i, c in enumerate(cons) if c[2] == "eq"]
    others = [i for i, c in enumerate(cons) if c[2] != "eq"]
    best = np.inf
    for sub in itertools.combinations(others, n - len(eqs)):
        idx = eqs + list(sub)
        A = np.array([cons[i][0] for i in idx]); b = np.array([cons[i][1] for i in idx])
        if abs(np.linalg.det(A)) < 1e-10:
            continue
        x = np.linalg.solve(A, b)
        ok = all((abs(r @ x - h) <= 1e-9) if kd == "eq" else (r @ x - h >= -1e-9)
                 for r, h, kd in cons)
        if ok:
            best = min(best, P.c @ x)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_solver_matches_vertex_enumeration(seed):
    rng = np.random.default_rng(100 + seed)
    n, m = 4, 3
    P = lpgen.random_lp(m, n, nnz_per_row=3, frac_ge=0.6, frac_free=0.0, seed=100 + seed)
    _, K = _norm_K(P)
    best = _vertex_enum(P, K)
    assert np.isfinite(best)
    lp = O.OracleLP.from_problem(P)
    tau, sig = _steps(P)
    for method in (0, 1, 2):
        r = O.solve(lp, O.Params(method=method, mem=3, tau=tau, sigma=sig), 200000, tol=1e-10,
                    kkt_every=1)
        assert r.status == 0, (method, r.iters)
        assert abs(P.c @ r.x - best) <= 1e-7 * (1 + abs(best)), (method, P.c @ r.x, best)
    del rng


def test_solver_matches_highs_on_tiny_workload():
    from scipy.optimize import linprog
    P = lpgen.tiny()
    _, K = _norm_K(P)
    res = linprog(P.c, A_eq=K, b_eq=P.q, bounds=list(zip(P.l, P.u)), method="highs")
    assert res.status == 0
    assert abs(res.fun - P.pobj_star) <= 1e-8 * (1 + abs(res.fun))
    lp = O.OracleLP.from_problem(P)
    tau, sig = _steps(P)
    r = O.solve(lp, O.Params(method=1, mem=10, tau=tau, sigma=sig), 50000, tol=1e-7,
                kkt_every=10)
    assert r.status == 0
    assert abs(P.c @ r.x - res.fun) <= 1e-5 * (1 + abs(res.fun))


# --------------------------------------------------------------------------
# The AA step equals Alg. 1 (standard type-II AA) when eta = 0, D-hat = I,
# beta = 1 and the projection is inactive (free variables, '=' rows)
# --------------------------------------------------------------------------
def _alg1_step(Fs, Us):
    """x+ = sum alpha_i F(u_i), alpha = argmin ||G alpha|| s.t. sum alpha = 1,
    solved through its KKT system with numpy."""
    G = np.stack([f - u for f, u in zip(Fs, Us)], axis=1)
    k = G.shape[1]
    A = np.zeros((k + 1, k + 1))
    A[:k, :k] = G.T @ G
    A[:k, k] = 1.0; A[k, :k] = 1.0
    rhs = np.zeros(k + 1); rhs[k] = 1.0
    sol = np.linalg.lstsq(A, rhs, rcond=None)[0]
    alpha = sol[:k]
    return np.stack(Fs, axis=1) @ alpha, alpha


def test_aa_step_equals_alg1():
    P = lpgen.random_lp(25, 25, nnz_per_row=5, frac_ge=0.0, frac_free=1.0, seed=7)
    lp = O.OracleLP.from_problem(P)
    tau, sig = _steps(P, 0.5)
    mem = 4
    prm = O.Params(method=1, mem=mem, tau=tau, sigma=sig, D=1e12, eta=0.0, beta=1.0,
                   dhat_mode=0)
    K_ITERS = 12
    r = O.solve(lp, prm, K_ITERS, trace=True, rec_len=K_ITERS + 1)
    assert np.all(r.branch[:K_ITERS] == 1)
    U = [np.zeros(P.n + P.m)] + list(r.rec_u)      # u^0, u^1, ..., u^{K}
    n = P.n

    def F(u):
        xh, yh = O.T(lp, tau, sig, u[:n], u[n:])
        return np.concatenate([xh, yh])

    checked = 0
    for k in range(1, K_ITERS):
        mk = min(mem, k)
        pts = U[k - mk:k + 1]
        x_alg1, alpha = _alg1_step([F(u) for u in pts], pts)
        err = np.linalg.norm(U[k + 1] - x_alg1) / np.linalg.norm(x_alg1)
        assert err < 1e-7, (k, err)
        # the H-form coefficients gamma telescope to alpha, and alpha sums to 1
        dG = np.stack([(F(pts[i + 1]) - pts[i + 1]) - (F(pts[i]) - pts[i])
                       for i in range(mk)], axis=1)
        rc, gam = O.aa_coeffs(dG, F(pts[-1]) - pts[-1], 0.0)
        assert rc == 0
        a = np.empty(mk + 1)
        a[0] = gam[0]
        a[1:mk] = gam[1:] - gam[:-1]
        a[mk] = 1.0 - gam[-1]
        assert abs(a.sum() - 1.0) < 1e-12
        assert np.allclose(a, alpha, rtol=1e-5, atol=1e-7)
        checked += 1
    assert checked == K_ITERS - 1


# --------------------------------------------------------------------------
# Where D-hat and beta enter the AA step (Alg. 2, the H-form H^k).  With
# H^k = -beta D-hat + (dU + beta D-hat dG)(dG'dG)^-1 dG' (eta = 0):
#   H^k dG = dU           (multi-secant: no D-hat, no beta)
#   H^k r  = -beta D-hat r for r orthogonal to span(dG).
# Both hold for any diagonal D-hat and any beta, so a D-hat placed on dU
# instead of dG, or a beta dropped from either term, breaks one of them.
# --------------------------------------------------------------------------
def _mix_case(seed, N=40, k=4):
    rng = np.random.default_rng(seed)
    dU = rng.standard_normal((N, k))
    dG = rng.standard_normal((N, k))
    dh = rng.uniform(0.3, 3.0, N)            # a diagonal D-hat far from I
    u = rng.standard_normal(N)
    return rng, dU, dG, dh, u


def _orth_to(dG, r):
    Q, _ = np.linalg.qr(dG)
    return r - Q @ (Q.T @ r)


def test_aa_mix_multisecant_with_dhat_and_beta():
    for seed in range(5):
        rng, dU, dG, dh, u = _mix_case(seed)
        w = rng.standard_normal(dG.shape[1])
        g = dG @ w                             # g^k in span(dG)
        rc, gam = O.aa_coeffs(dG, g, 0.0)
        assert rc == 0 and np.allclose(gam, w, rtol=0, atol=1e-11)
        for beta in (0.5, 0.25, 1.0):
            step = O.aa_mix(u, g, dU, dG, dh, beta, gam)
            assert np.allclose(step, u - dU @ w, rtol=0, atol=1e-10), (seed, beta)


def test_aa_mix_residual_orthogonal_to_history():
    for seed in range(5):
        rng, dU, dG, dh, u = _mix_case(seed)
        g = _orth_to(dG, rng.standard_normal(dG.shape[0]))
        rc, gam = O.aa_coeffs(dG, g, 0.0)
        assert rc == 0 and np.max(np.abs(gam)) < 1e-12
        for beta in (0.5, 0.25, 1.0):
            step = O.aa_mix(u, g, dU, dG, dh, beta, gam)
            assert np.allclose(step, u + beta * dh * g, rtol=0, atol=1e-12), (seed, beta)


def test_aa_mix_general_residual():
    # g = dG w + r with r orthogonal to span(dG): u - H g = u - dU w + beta D-hat r
    for seed in range(5):
        rng, dU, dG, dh, u = _mix_case(seed, N=60, k=6)
        w = rng.standard_normal(dG.shape[1])
        r = _orth_to(dG, rng.standard_normal(dG.shape[0]))
        g = dG @ w + r
        rc, gam = O.aa_coeffs(dG, g, 0.0)
        assert rc == 0
        step = O.aa_mix(u, g, dU, dG, dh, 0.5, gam)
        assert np.allclose(step, u - dU @ w + 0.5 * dh * r, rtol=0, atol=1e-10), seed


def test_solver_aa_steps_with_dhat_and_beta():
    """Every AA step of the oracle's solver, with the D-hat of the Remark
    (not I), beta = 0.5 and eta = 0, on an LP whose projection is inactive
    (free variables, '=' rows): splitting g^k = dG gamma + r with numpy's
    least squares, the step must be u^{k+1} - u^k = -dU gamma + beta D-hat r."""
    P = lpgen.random_lp(25, 25, nnz_per_row=5, frac_ge=0.0, frac_free=1.0, seed=7)
    lp = O.OracleLP.from_problem(P)
    tau, sig = _steps(P, 0.5)
    mem, beta = 4, 0.5
    prm = O.Params(method=1, mem=mem, tau=tau, sigma=sig, D=1e12, eta=0.0, beta=beta,
                   dhat_mode=1)
    K_ITERS = 10
    r = O.solve(lp, prm, K_ITERS, trace=True, rec_len=K_ITERS + 1)
    assert np.all(r.branch[:K_ITERS] == 1)
    dx, dy = O.dhat(lp, 1)
    dh = np.concatenate([dx, dy])
    assert np.ptp(dh) > 0.1                       # D-hat is not a multiple of I here
    U = [np.zeros(P.n + P.m)] + list(r.rec_u)     # u^0 .. u^K
    n = P.n

    def G(u):
        xh, yh = O.T(lp, tau, sig, u[:n], u[n:])
        return np.concatenate([xh, yh]) - u

    for k in range(1, K_ITERS):
        mk = min(mem, k)
        dU = np.stack([U[i + 1] - U[i] for i in range(k - mk, k)], axis=1)
        dG = np.stack([G(U[i + 1]) - G(U[i]) for i in range(k - mk, k)], axis=1)
        g = G(U[k])
        gam = np.linalg.lstsq(dG, g, rcond=None)[0]
        res = g - dG @ gam
        want = U[k] - dU @ gam + beta * dh * res
        err = np.linalg.norm(U[k + 1] - want) / np.linalg.norm(want)
        assert err < 1e-7, (k, err)


# --------------------------------------------------------------------------
# Least-squares kernels: library cross-checks and the Tikhonov bound
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 3, 8])
def test_aa_coeffs_library_and_bound(k):
    rng = np.random.default_rng(k)
    N = 200
    dG = rng.standard_normal((N, k)) * rng.lognormal(0, 2, k)
    g = rng.standard_normal(N)
    for eta in (1e-10, 1e-2, 10.0):
        rc, gam = O.aa_coeffs(dG, g, eta)
        assert rc == 0
        ref = np.linalg.solve(dG.T @ dG + eta * np.eye(k), dG.T @ g)
        assert np.allclose(gam, ref, rtol=1e-8, atol=1e-12)
        # ||(G'G + eta I)^-1 G'|| <= 1 / (2 sqrt(eta))  (Sec. 5.2)
        assert np.linalg.norm(gam) <= np.linalg.norm(g) / (2 * np.sqrt(eta)) * (1 + 1e-12)
    rc, gam = O.aa_coeffs(dG, g, 0.0)
    assert np.allclose(gam, np.linalg.lstsq(dG, g, rcond=None)[0], rtol=1e-7)


def test_aa_coeffs_reports_singular_gram():
    # rank one with exactly representable Gram [[16, 32], [32, 64]]: the second pivot
    # is exactly 0, so with eta = 0 the factorisation must fail (reading R4)
    dG = np.stack([np.ones(16), 2 * np.ones(16)], axis=1)
    rc, _ = O.aa_coeffs(dG, np.ones(16), 0.0)
    assert rc != 0


def test_qr_coeffs_equal_lstsq():
    rng = np.random.default_rng(3)
    dG = rng.standard_normal((50, 5))
    g = rng.standard_normal(50)
    rc, gam = O.qr_coeffs(dG, g)
    assert rc == 0 and np.allclose(gam, np.linalg.lstsq(dG, g, rcond=None)[0], rtol=1e-10)


# --------------------------------------------------------------------------
# FAA filters (Alg. 4, 5, 6; Lemma 1.1, Proposition 1.2 and the conditioning
# lemma of Sec. 4)
# --------------------------------------------------------------------------
def _cols_with_sines(sines, N=6):
    """Columns f_1.. (newest first) where f_i has sine exactly s_i to span(f_1..f_{i-1})."""
    cols = [np.eye(N)[0]]
    for i, s in enumerate(sines, start=1):
        c = np.sqrt(1 - s * s)
        cols.append(c * np.eye(N)[0] + s * np.eye(N)[i])
    return np.stack(cols, axis=1)


def test_angle_filter_by_hand():
    # newest-first columns with sines 0.5, 0.1, 0.9 -> the 0.1 one is dropped at c_s = 0.2
    Fr = _cols_with_sines([0.5, 0.1, 0.9])
    F = Fr[:, ::-1]                          # oldest first, as the solver stores them
    E = np.eye(6)[:, :4]
    keep = O.faa_filter(E, F, 0.2, 1e30)
    # reversed index 2 (sine 0.1) is oldest-first index 4 - 1 - 2 = 1
    assert keep.tolist() == [True, False, True, True]
    # threshold just below / above a sine decides
    assert O.faa_filter(E, F, 0.09, 1e30).tolist() == [True, True, True, True]
    # c_s = 0.51 drops the sines 0.5 and 0.1 (oldest-first indices 2 and 1); the 0.9 one
    # (oldest-first index 0) and the newest column survive
    assert O.faa_filter(E, F, 0.51, 1e30).tolist() == [True, False, False, True]


def test_angle_filter_keeps_newest_and_drops_duplicate():
    rng = np.random.default_rng(0)
    F = rng.standard_normal((30, 4))
    F[:, 1] = F[:, 3]                        # an older copy of the newest column
    keep = O.faa_filter(rng.standard_normal((30, 4)), F, 0.2, 1e30)
    assert keep[3] and not keep[1] and keep[0] and keep[2]


def test_length_bounds_by_hand_and_prop12():
    c_s = 0.2
    c_t = np.sqrt(1 - c_s ** 2)
    b = O.length_bounds([2.0, 4.0], c_s)
    assert b[0] == pytest.approx(1 / 4)
    assert b[1] == pytest.approx((c_t ** 2 / 4 + 1 / 16) / c_s ** 2)
    # Proposition 1.2 on F meeting the lemma's hypotheses: ||col j of R^-1||^2 <= b_j
    rng = np.random.default_rng(1)
    for trial in range(20):
        k = 5
        Q = np.linalg.qr(rng.standard_normal((40, k)))[0]
        F = Q @ np.triu(rng.uniform(0.5, 1.5, (k, k)) * np.where(np.eye(k) > 0, 1.0, 0.3))
        F *= rng.lognormal(0, 1, k)
        Rq = np.linalg.qr(F, mode="r")
        fn = np.linalg.norm(F, axis=0)
        sines = np.abs(np.diag(Rq)) / fn
        cos_ok = all(abs(F[:, i] @ F[:, j]) / (fn[i] * fn[j]) <= np.sqrt(1 - c_s ** 2)
                     for i in range(k) for j in range(i))
        if sines[1:].min() < c_s or not cos_ok:
            continue
        S = np.linalg.inv(Rq)
        bb = O.length_bounds(fn, c_s)
        assert np.all(np.sum(S * S, axis=0) <= bb * (1 + 1e-12)), trial


def test_prop12_tight_case_with_small_middle_column():
    # f1 = e1, f2 = 1e-3 (c_t e1 + c_s e2), f3 = c_t e2 + c_s e3 meet Lemma 1.1's
    # hypotheses (every sine to the earlier span is c_s, every cosine <= c_t); the small
    # f2 makes column 3 of R^-1 large, and only the i = 2 term of b_3 covers it.
    c_s = 0.5
    c_t = np.sqrt(1 - c_s ** 2)
    e = np.eye(5)
    F = np.stack([e[0], 1e-3 * (c_t * e[0] + c_s * e[1]), c_t * e[1] + c_s * e[2]], axis=1)
    R = np.linalg.qr(F, mode="r")
    S = np.linalg.inv(R)
    s2 = np.sum(S * S, axis=0)
    b = O.length_bounds(np.linalg.norm(F, axis=0), c_s)
    assert np.all(s2 <= b * (1 + 1e-12))
    assert s2[2] > 0.99 * b[2]            # the bound is nearly attained here


def test_length_filter_keeps_newest_prefix_and_bound():
    # orthonormal F (sines 1), unit E columns: b_j from the formula; kappa chosen so
    # that exactly the two newest columns survive
    N, k = 12, 4
    F = np.eye(N)[:, :k]
    E = np.eye(N)[:, :k]
    c_s = 0.2
    b = O.length_bounds(np.ones(k), c_s)
    C2 = 2 * (b[0] + b[1])
    C3 = 3 * (b[0] + b[1] + b[2])
    kappa = np.sqrt((C2 + C3) / 2)
    keep = O.faa_filter(E, F, c_s, kappa)
    assert keep.tolist() == [False, False, True, True]       # newest two (oldest first)
    # the conditioning lemma: ||E||_F^2 ||R^-1||_F^2 <= kappa^2 on what survives
    R = np.linalg.qr(F[:, keep], mode="r")
    assert np.sum(E[:, keep] ** 2) * np.sum(np.linalg.inv(R) ** 2) <= kappa ** 2
    # no prefix passes -> nothing kept (reading R7)
    assert not O.faa_filter(E, F, c_s, 1e-3).any()


def test_conditioning_lemma_random():
    rng = np.random.default_rng(2)
    hits = 0
    for trial in range(40):
        N, k = 60, 6
        F = rng.standard_normal((N, k)) * rng.lognormal(0, 2, k)
        E = rng.standard_normal((N, k)) * rng.lognormal(0, 2, k)
        kappa = 10 ** rng.uniform(0, 3)
        keep = O.faa_filter(E, F, 0.2, kappa)
        if not keep.any():
            continue
        # hypotheses of Lemma 1.1 (pairwise cosines) must hold for the bound to apply
        Fk = F[:, keep][:, ::-1]
        fn = np.linalg.norm(Fk, axis=0)
        cos = np.abs(Fk.T @ Fk) / np.outer(fn, fn)
        if np.max(cos - np.eye(len(fn))) > np.sqrt(1 - 0.04):
            continue
        R = np.linalg.qr(Fk, mode="r")
        val = np.sum(E[:, keep] ** 2) * np.sum(np.linalg.inv(R) ** 2)
        assert val <= kappa ** 2 * (1 + 1e-9), (trial, val, kappa ** 2)
        hits += 1
    assert hits >= 10


# --------------------------------------------------------------------------
# Safeguard and counters (Alg. 2)
# --------------------------------------------------------------------------
def test_safeguard_extremes_and_counters():
    P = lpgen.random_lp(40, 60, seed=11)
    lp = O.OracleLP.from_problem(P)
    tau, sig = _steps(P)
    base = O.solve(lp, O.Params(method=0, mem=0, tau=tau, sigma=sig), 300, rec_len=301)
    # D tiny: the AA step is never taken; iterates are plain PDHG bit for bit
    r = O.solve(lp, O.Params(method=1, mem=5, tau=tau, sigma=sig, D=1e-300), 300, rec_len=301,
                trace=True)
    assert r.aa_steps == 0 and r.pdhg_steps == 300
    assert np.array_equal(r.rec_u, base.rec_u)
    # memory 0: no AA step possible
    r0 = O.solve(lp, O.Params(method=1, mem=0, tau=tau, sigma=sig, D=1e300), 300, rec_len=301)
    assert r0.aa_steps == 0 and np.array_equal(r0.rec_u, base.rec_u)
    # D huge: every step accepted
    r = O.solve(lp, O.Params(method=1, mem=5, tau=tau, sigma=sig, D=1e300), 50, trace=True)
    assert r.aa_steps == 50 and r.pdhg_steps == 0
    # every decision of a normal run obeys the threshold with i counted along the way
    for cdiv in (1.0, 3.0):
        prm = O.Params(method=1, mem=5, tau=tau, sigma=sig, D=1.0, c_div=cdiv)
        r = O.solve(lp, prm, 400, trace=True)
        g0 = np.linalg.norm(np.concatenate(O.T(lp, tau, sig, np.clip(0, P.l, P.u),
                                                   np.zeros(P.m))) -
                            np.concatenate([np.clip(0, P.l, P.u), np.zeros(P.m)]))
        i = 0
        for t in range(400):
            ok = r.gnorm[t] <= g0 * (i / cdiv + 1) ** -2.0
            assert (r.branch[t] == 1) == ok or r.branch[t] == 2
            i += r.branch[t] == 1
        assert i == r.aa_steps and r.aa_steps + r.pdhg_steps == 400


def test_faa_with_no_kept_columns_is_pdhg():
    # LengthFilter keeping nothing gives H = -beta D-hat: with D-hat = I, beta = 1 the
    # step is P(u + g) = T u (up to rounding of u + (Tu - u))
    P = lpgen.random_lp(40, 60, seed=12)
    lp = O.OracleLP.from_problem(P)
    tau, sig = _steps(P)
    base = O.solve(lp, O.Params(method=0, mem=0, tau=tau, sigma=sig), 100, rec_len=101)
    r = O.solve(lp, O.Params(method=2, mem=5, tau=tau, sigma=sig, D=1e300, kappa=1e-300,
                             dhat_mode=0), 100, rec_len=101, trace=True)
    assert r.aa_steps == 100 and np.all(r.mk == 0)
    assert np.max(np.abs(r.rec_u - base.rec_u)) < 1e-12 * (1 + np.max(np.abs(base.rec_u)))


def test_faa_adaptive_memory_shrinks():
    P = lpgen.tiny()
    lp = O.OracleLP.from_problem(P)
    tau, sig = _steps(P)
    r = O.solve(lp, O.Params(method=2, mem=5, tau=tau, sigma=sig, D=10), 600, trace=True)
    used = r.mk[r.branch == 1]
    assert used.size > 0 and used.max() <= 5
    assert (used < 5).any()   # filtering dropped columns at least once


# --------------------------------------------------------------------------
# Preconditioning (Sec. 5.2 set-up: Ruiz x10 + Pock-Chambolle, reading R12)
# --------------------------------------------------------------------------
def test_pock_chambolle_by_hand():
    # K = [[4, 0], [1, 9]]: row sums 4, 10; column sums 5, 9
    P = lpgen.from_dense([[4.0, 0.0], [1.0, 9.0]], [0, 0], [1, 1], [1, 1], [0, 0], [1, 1])
    dr, dc = O.scaling(O.OracleLP.from_problem(P), 0, True)
    assert np.allclose(dr, [0.5, 1 / np.sqrt(10)], rtol=1e-15)
    assert np.allclose(dc, [1 / np.sqrt(5), 1 / 3], rtol=1e-15)


def test_one_ruiz_pass_by_hand():
    # K = [[4, 1], [0, 9]]: row maxima 4, 9 and column maxima 4, 9 of the same
    # matrix give D_r = D_c = (1/2, 1/3).  (Taking the column maxima from the
    # row-scaled matrix would give D_c = (1/sqrt 2, 1/sqrt 3).)
    P = lpgen.from_dense([[4.0, 1.0], [0.0, 9.0]], [0, 0], [1, 1], [1, 1], [0, 0], [1, 1])
    dr, dc = O.scaling(O.OracleLP.from_problem(P), 1, False)
    assert np.allclose(dr, [0.5, 1 / 3], rtol=1e-15)
    assert np.allclose(dc, [0.5, 1 / 3], rtol=1e-15)
    # an empty row or column keeps the factor 1
    Q = lpgen.from_dense([[4.0, 0.0], [0.0, 0.0]], [0, 0], [1, 1], [1, 1], [0, 0], [1, 1])
    dr, dc = O.scaling(O.OracleLP.from_problem(Q), 3, False)
    assert np.allclose(dr, [0.5, 1.0], rtol=1e-15)
    assert np.allclose(dc, [0.5, 1.0], rtol=1e-15)


def test_ruiz_equilibrates_inf_norms():
    P = lpgen.random_lp(60, 90, nnz_per_row=6, row_scale_sigma=3.0, seed=4)
    lp = O.OracleLP.from_problem(P)
    dr, dc = O.scaling(lp, 40, False)
    S = O.scaled_lp(lp, dr, dc)
    import scipy.sparse as sp
    A = abs(sp.csr_matrix((S.v, S.ci.astype(np.int64), S.rp), shape=(P.m, P.n)))
    rmax = A.max(axis=1).toarray().ravel()
    cmax = A.max(axis=0).toarray().ravel()
    assert np.max(np.abs(rmax[rmax > 0] - 1)) < 1e-3
    assert np.max(np.abs(cmax[cmax > 0] - 1)) < 1e-3


def test_scaled_lp_has_the_same_solution():
    P = lpgen.random_lp(40, 70, nnz_per_row=5, frac_ge=0.4, frac_free=0.1,
                        frac_lower_only=0.1, frac_upper_only=0.1, row_scale_sigma=2.0, seed=8)
    lp = O.OracleLP.from_problem(P)
    dr, dc = O.scaling(lp, 10, True)
    S = O.scaled_lp(lp, dr, dc)
    # the constructed optimum maps to an optimum of the scaled LP
    k = O.kkt(S, P.x_star / dc, P.y_star / dr)
    assert k["r_p"] < 1e-12 and k["r_d"] < 1e-12 and abs(k["pobj"] - P.pobj_star) < 1e-9
    # and solving the scaled LP gives the original optimum back
    import scipy.sparse as sp
    A = sp.csr_matrix((S.v, S.ci.astype(np.int64), S.rp), shape=(P.m, P.n)).toarray()
    step = 0.9 / np.linalg.norm(A, 2)
    r = O.solve(S, O.Params(method=1, mem=5, tau=step, sigma=step), 300000, tol=3e-5, kkt_every=10)
    assert r.status == 0
    x = dc * r.x
    assert abs(P.c @ x - P.pobj_star) <= 1e-3 * (1 + abs(P.pobj_star))
    assert O.kkt(lp, x, dr * r.y)["kkt"] < 1e-3
