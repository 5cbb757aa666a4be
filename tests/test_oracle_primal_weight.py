"""Pins of the oracle's primal weight update (Alg. "Primal weight update" and
the Remark on its form; readings R13-R15), CPU only.

Each pin composes runs of the oracle *without* the update: a run to u^K,
then a fresh run started from u^K with the steps (and D-hat) the update must
produce.  Since PDHG gives u^{k+1} = T(u^k), and a fresh run's first step is a
plain T step with an empty memory (exactly what R15 makes the update
iteration), the run with the update must equal the composition iterate by
iterate.  This checks when the update happens, which iterate the change is
measured from, the omega formula, which step gets 1/omega and which omega,
the memory reset, and which alpha the D-hat blend picks.
"""
import numpy as np
import pytest

import lpgen
from oracle import oracle as O

K = 40


def _lp():
    P = lpgen.random_lp(60, 150, nnz_per_row=5, frac_ge=0.3, frac_free=0.1, seed=21)
    return P, O.OracleLP.from_problem(P)


def _fresh(lp, P, u_start, prm, iters):
    return O.solve(lp, prm, iters, x0=u_start[:P.n], y0=u_start[P.n:], rec_len=iters)


@pytest.mark.parametrize("theta,tau,sigma", [(1.0, 0.05, 0.05), (0.5, 0.02, 0.1)])
def test_omega_update_and_step_assignment(theta, tau, sigma):
    P, lp = _lp()
    base = O.Params(method=0, mem=0, tau=tau, sigma=sigma)
    pw = O.Params(method=0, mem=0, tau=tau, sigma=sigma, pw_period=K, pw_theta=theta, pw_dhat=0)
    run1 = O.solve(lp, pw, 2 * K, rec_len=2 * K)
    run2 = O.solve(lp, base, K, rec_len=K)
    u0 = np.concatenate([np.clip(np.zeros(P.n), P.l, P.u), np.zeros(P.m)])
    uK = run2.rec_u[K - 1]                                  # rec_u[j] = u^{j+1}
    assert np.array_equal(run1.rec_u[:K], run2.rec_u[:K])   # nothing changes before k = K
    dx = np.linalg.norm(uK[:P.n] - u0[:P.n])
    dy = np.linalg.norm(uK[P.n:] - u0[P.n:])
    gamma, w0 = np.sqrt(tau * sigma), np.sqrt(sigma / tau)
    w1 = np.exp(theta * np.log(dy / dx) + (1 - theta) * np.log(w0))
    run3 = _fresh(lp, P, uK, O.Params(method=0, mem=0, tau=gamma / w1, sigma=gamma * w1), K - 1)
    for j in range(K - 1):
        r = run1.rec_u[K + j]
        assert np.linalg.norm(r - run3.rec_u[j]) <= 1e-12 * np.linalg.norm(r), j


def test_update_is_skipped_when_a_block_does_not_move():
    # no constraints: y is empty, Delta_y = 0 <= eps_zero, omega never changes
    n = 20
    rng = np.random.default_rng(3)
    P = lpgen.Problem(0, n, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0),
                      np.zeros(0, np.int8), np.zeros(0), rng.standard_normal(n),
                      -np.ones(n), np.ones(n))
    lp = O.OracleLP.from_problem(P)
    a = O.solve(lp, O.Params(method=1, mem=3, tau=0.3, sigma=0.3), 30, rec_len=30)
    b = O.solve(lp, O.Params(method=1, mem=3, tau=0.3, sigma=0.3, pw_period=5), 30, rec_len=30)
    assert np.array_equal(a.rec_u, b.rec_u)


def test_memory_reset_restarts_anderson():
    # theta = 0 keeps omega (and T); the update only resets the memory, so the
    # AA run after u^K is a fresh AA run from u^K (safeguard always open)
    P, lp = _lp()
    kw = dict(method=1, mem=5, tau=0.05, sigma=0.05, D=1e30)
    run1 = O.solve(lp, O.Params(**kw, pw_period=K, pw_theta=0.0, pw_dhat=0), 2 * K, rec_len=2 * K,
                   trace=True)
    run2 = O.solve(lp, O.Params(**kw), K, rec_len=K)
    run3 = _fresh(lp, P, run2.rec_u[K - 1], O.Params(**kw), K - 1)
    assert run1.branch[K - 1] == 0                          # the update iteration: a plain step
    for j in range(K - 1):
        r = run1.rec_u[K + j]
        assert np.linalg.norm(r - run3.rec_u[j]) <= 1e-11 * np.linalg.norm(r), j
    # without the reset the runs part
    run4 = O.solve(lp, O.Params(**kw), 2 * K, rec_len=2 * K)
    assert np.linalg.norm(run4.rec_u[K + 5] - run1.rec_u[K + 5]) > 1e-6


@pytest.mark.parametrize("rho_min", [-1.0, 1e9])
def test_dhat_blend_picks_alpha_by_residual_decrease(rho_min):
    # omega stays 1 (theta = 0, tau = sigma), so the blend is
    # (1 - alpha) I + alpha D-hat_base: with alpha_dec = 0 and alpha_inc = 1 the
    # run after u^K must equal a fresh run with D-hat = I (decrease deemed
    # sufficient) or with the base D-hat (deemed insufficient)
    P, lp = _lp()
    kw = dict(method=1, mem=5, tau=0.05, sigma=0.05, D=1e30)
    run1 = O.solve(lp, O.Params(**kw, pw_period=K, pw_theta=0.0, pw_dhat=1, pw_rho_min=rho_min,
                                pw_alpha_dec=0.0, pw_alpha_inc=1.0), 2 * K, rec_len=2 * K)
    run2 = O.solve(lp, O.Params(**kw), K, rec_len=K, trace=True)
    r1, r2 = run2.gnorm[K - 1], run2.gnorm[K - 2]           # ||g^{K-1}||, ||g^{K-2}||
    rho = (r2 - r1) / max(r2, 1e-10)
    dhat_mode = 0 if rho >= rho_min else 1
    assert dhat_mode == (0 if rho_min < 0 else 1)
    run3 = _fresh(lp, P, run2.rec_u[K - 1], O.Params(**kw, dhat_mode=dhat_mode), K - 1)
    for j in range(K - 1):
        r = run1.rec_u[K + j]
        assert np.linalg.norm(r - run3.rec_u[j]) <= 1e-11 * np.linalg.norm(r), (j, dhat_mode)


def test_second_update_measures_from_the_first():
    # two updates (k = K and 2K): the second measures the change from u^K
    P, lp = _lp()
    gamma = 0.05
    pw = O.Params(method=0, mem=0, tau=gamma, sigma=gamma, pw_period=K, pw_theta=1.0, pw_dhat=0)
    run1 = O.solve(lp, pw, 3 * K, rec_len=3 * K)
    u0 = np.concatenate([np.clip(np.zeros(P.n), P.l, P.u), np.zeros(P.m)])
    us = [u0]
    seg = O.solve(lp, O.Params(method=0, mem=0, tau=gamma, sigma=gamma), K, rec_len=K)
    us.append(seg.rec_u[K - 1])                               # u^K
    for stage in range(2):
        a, b = us[-2], us[-1]
        w = np.linalg.norm(b[P.n:] - a[P.n:]) / np.linalg.norm(b[:P.n] - a[:P.n])
        seg = _fresh(lp, P, b, O.Params(method=0, mem=0, tau=gamma / w, sigma=gamma * w), K)
        us.append(seg.rec_u[K - 1])                           # u^{(stage + 2) K}
    for j in range(K - 1):
        r = run1.rec_u[2 * K + j]
        assert np.linalg.norm(r - seg.rec_u[j]) <= 1e-11 * np.linalg.norm(r), j


@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_dhat_blend_scales_x_by_one_over_omega_and_y_by_omega(alpha):
    # after one update with theta = 1: omega = Delta_y / Delta_x (computed here
    # from a run without the update), and the D-hat in use must be
    # (1 - alpha) diag(1/omega, omega) + alpha diag(D1/omega, D2 omega)
    P, lp = _lp()
    gamma = 0.05
    run1 = O.solve(lp, O.Params(method=1, mem=4, tau=gamma, sigma=gamma, pw_period=K,
                                pw_theta=1.0, pw_dhat=1, pw_alpha_dec=alpha, pw_alpha_inc=alpha),
                   K + 5)
    seg = O.solve(lp, O.Params(method=1, mem=4, tau=gamma, sigma=gamma), K, rec_len=K)
    u0 = np.concatenate([np.clip(np.zeros(P.n), P.l, P.u), np.zeros(P.m)])
    uK = seg.rec_u[K - 1]
    w = np.linalg.norm(uK[P.n:] - u0[P.n:]) / np.linalg.norm(uK[:P.n] - u0[:P.n])
    d1, d2 = O.dhat(lp, 1)
    want = np.concatenate([((1 - alpha) + alpha * d1) / w, ((1 - alpha) + alpha * d2) * w])
    assert np.allclose(run1.dhat, want, rtol=1e-12, atol=0)
