"""Seeded synthetic LP generators shared by the tests, the oracle and the CUDA path.

Every LP is feasible by construction with a known primal-dual optimum
(x*, y*, lambda*): the constraint data q and the costs c are derived from a
drawn optimum so that primal feasibility, dual feasibility (c - K'y* = lambda*
with lambda* in Lambda, y* >= 0 on '>=' rows) and complementary slackness hold
exactly in real arithmetic.  This module draws numbers and assembles CSR
arrays; it holds none of the solver's arithmetic.

LP form (Sec. 2.1, eq. LP-O): min c'x s.t. Gx >= h, Ax = b, l <= x <= u, with
K = [G; A] stored as one CSR matrix and a sense byte per row (1: '>=', 0: '=').

Workloads (sizes and distributions of the benchmark configurations):
  tiny    200 x 500, 10 nnz per row at distinct uniform columns, N(0,1) values,
          all '=' rows, 0 <= x <= 10.
  medium  100k x 300k, log-normal row lengths (median 7, sigma 1.45, clipped to
          [1, 2000]; mean about 20, Z about 2M), values N(0,1) times one
          lognormal(0,2) scale per row, 70% '=' / 30% '>=' rows, bounds
          [0, U(1,100)] with 10% free variables.
  large   2M x 5M, Chung-Lu power-law row and column degrees (exponent 2.1)
          scaled to Z about 50M with duplicates removed, values N(0,1) times one
          lognormal(0,3) scale per row, 20% '>=' rows, bounds as medium.
  banded  the large sizes (2M x 5M, Z = 50M) with local structure: row i holds
          the 25 consecutive columns from floor(i (n - 25) / (m - 1)); values,
          senses and bounds as large.  A diagnostic of the half-steps' streaming
          ceiling (the gathered entries of a row share cache lines), not a
          workload of the paper's kind.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20250800


@dataclass
class Problem:
    m: int
    n: int
    row_ptr: np.ndarray      # int64 (m + 1)
    col_idx: np.ndarray      # int32 (nnz)
    val: np.ndarray          # float64 (nnz)
    sense: np.ndarray        # int8 (m): 1 '>=' row, 0 '=' row
    q: np.ndarray            # float64 (m)
    c: np.ndarray            # float64 (n)
    l: np.ndarray            # float64 (n), may hold -inf
    u: np.ndarray            # float64 (n), may hold +inf
    x_star: np.ndarray | None = None
    y_star: np.ndarray | None = None
    lam_star: np.ndarray | None = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def pobj_star(self) -> float:
        return float(self.c @ self.x_star)

    def csr_matvec(self, x):
        """K x by a library sparse routine (input assembly only)."""
        return _csr(self) @ x

    def csr_rmatvec(self, y):
        return _csr(self).T @ y


def _csr(P: Problem):
    import scipy.sparse as sp
    return sp.csr_matrix((P.val, P.col_idx.astype(np.int64), P.row_ptr), shape=(P.m, P.n))


def _csr_from_coo(m, rows, cols, vals):
    """Sort (row, col) pairs, drop repeated pairs, return CSR arrays."""
    key = rows.astype(np.int64) * (np.int64(1) << 32) + cols.astype(np.int64)
    order = np.argsort(key, kind="stable")
    key = key[order]
    keep = np.ones(len(key), dtype=bool)
    keep[1:] = key[1:] != key[:-1]
    order = order[keep]
    r = rows[order]; c = cols[order]; v = vals[order]
    counts = np.bincount(r, minlength=m)
    rp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rp[1:])
    return rp, c.astype(np.int32), v.astype(np.float64)


def construct(rng, m, n, row_ptr, col_idx, val, sense, l, u, name="", meta=None) -> Problem:
    """Draw an optimum (x*, y*, lambda*) and derive q, c from it.

    x*: a variable with a finite bound sits on a bound with probability 1/2
        (lower/upper evenly when both are finite), else strictly inside
        (U(l, u) when boxed, bound + Exp(1) when one-sided); free: N(0, 1).
    y*: '>=' rows active with y* ~ U(0.1, 1) or inactive with y* = 0 (1/2 each);
        '=' rows y* ~ N(0, 1).
    q:  (K x*)_i on '=' and active rows, (K x*)_i - U(0.1, 1) on inactive rows.
    lambda*: U(0.1, 1) at a lower bound, -U(0.1, 1) at an upper bound, else 0.
    c = K' y* + lambda*.
    """
    P = Problem(m, n, row_ptr, col_idx, val, np.asarray(sense, dtype=np.int8),
                np.zeros(m), np.zeros(n), np.asarray(l, dtype=np.float64),
                np.asarray(u, dtype=np.float64), name=name, meta=meta or {})
    lf, uf = np.isfinite(P.l), np.isfinite(P.u)
    x = np.zeros(n)
    lam = np.zeros(n)
    at_bound = rng.random(n) < 0.5
    pick_upper = rng.random(n) < 0.5
    mag = rng.uniform(0.1, 1.0, n)
    boxed = lf & uf
    lower_only = lf & ~uf
    upper_only = ~lf & uf
    free = ~lf & ~uf
    # boxed
    b_lo = boxed & at_bound & ~pick_upper
    b_up = boxed & at_bound & pick_upper
    b_in = boxed & ~at_bound
    x[b_lo] = P.l[b_lo]; lam[b_lo] = mag[b_lo]
    x[b_up] = P.u[b_up]; lam[b_up] = -mag[b_up]
    x[b_in] = rng.uniform(P.l[b_in], P.u[b_in])
    # one-sided
    lo_at = lower_only & at_bound
    lo_in = lower_only & ~at_bound
    x[lo_at] = P.l[lo_at]; lam[lo_at] = mag[lo_at]
    x[lo_in] = P.l[lo_in] + rng.exponential(1.0, int(lo_in.sum()))
    up_at = upper_only & at_bound
    up_in = upper_only & ~at_bound
    x[up_at] = P.u[up_at]; lam[up_at] = -mag[up_at]
    x[up_in] = P.u[up_in] - rng.exponential(1.0, int(up_in.sum()))
    x[free] = rng.standard_normal(int(free.sum()))

    ge = P.sense == 1
    active = rng.random(m) < 0.5
    y = np.zeros(m)
    y[~ge] = rng.standard_normal(int((~ge).sum()))
    ya = ge & active
    y[ya] = rng.uniform(0.1, 1.0, int(ya.sum()))
    slack = np.where(ge & ~active, rng.uniform(0.1, 1.0, m), 0.0)
    P.q = P.csr_matvec(x) - slack
    P.c = P.csr_rmatvec(y) + lam
    P.x_star, P.y_star, P.lam_star = x, y, lam
    return P


def _bounds_medium(rng, n):
    """[0, U(1, 100)] bounds, 10% free variables."""
    l = np.zeros(n)
    u = rng.uniform(1.0, 100.0, n)
    free = rng.random(n) < 0.10
    l[free] = -np.inf
    u[free] = np.inf
    return l, u


def random_lp(m, n, nnz_per_row=5, frac_ge=0.3, frac_free=0.1, frac_lower_only=0.0,
              frac_upper_only=0.0, row_scale_sigma=0.0, seed=0, name="random") -> Problem:
    """Small general-purpose LP for tests: row lengths Poisson(nnz_per_row) >= 1
    (capped at n), distinct uniform columns, N(0,1) values times a per-row
    lognormal(0, row_scale_sigma) scale, mixed senses and bound kinds."""
    rng = np.random.default_rng(seed)
    lens = np.clip(rng.poisson(nnz_per_row, m), 1, max(1, n)) if n > 0 else np.zeros(m, int)
    rows = np.repeat(np.arange(m), lens)
    cols = np.concatenate([rng.choice(n, k, replace=False) for k in lens]) if m and n else \
        np.zeros(0, np.int64)
    vals = rng.standard_normal(len(rows))
    if row_scale_sigma > 0:
        vals *= np.exp(rng.normal(0.0, row_scale_sigma, m))[rows]
    rp, ci, v = _csr_from_coo(m, rows, cols, vals)
    sense = (rng.random(m) < frac_ge).astype(np.int8)
    l = np.zeros(n); u = rng.uniform(1.0, 10.0, n)
    kind = rng.random(n)
    t0 = frac_free; t1 = t0 + frac_lower_only; t2 = t1 + frac_upper_only
    fr = kind < t0
    lo = (kind >= t0) & (kind < t1)
    up = (kind >= t1) & (kind < t2)
    l[fr] = -np.inf; u[fr] = np.inf
    u[lo] = np.inf
    l[up] = -np.inf
    return construct(rng, m, n, rp, ci, v, sense, l, u, name=name)


def tiny(seed=SEED_BASE + 1) -> Problem:
    """200 x 500, 10 nnz per row at distinct uniform columns, N(0,1), all '=' rows,
    0 <= x <= 10."""
    m, n, k = 200, 500, 10
    rng = np.random.default_rng(seed)
    rows = np.repeat(np.arange(m), k)
    cols = np.concatenate([rng.choice(n, k, replace=False) for _ in range(m)])
    vals = rng.standard_normal(m * k)
    rp, ci, v = _csr_from_coo(m, rows, cols, vals)
    return construct(rng, m, n, rp, ci, v, np.zeros(m, np.int8), np.zeros(n),
                     np.full(n, 10.0), name="tiny-200x500")


def medium(seed=SEED_BASE + 2, m=100_000, n=300_000) -> Problem:
    """100k x 300k, Z about 2M (see module docstring)."""
    rng = np.random.default_rng(seed)
    lens = np.rint(rng.lognormal(np.log(7.0), 1.45, m)).astype(np.int64)
    lens = np.clip(lens, 1, min(2000, n))
    rows = np.repeat(np.arange(m, dtype=np.int64), lens)
    cols = rng.integers(0, n, len(rows))
    vals = rng.standard_normal(len(rows)) * np.exp(rng.normal(0.0, 2.0, m))[rows]
    rp, ci, v = _csr_from_coo(m, rows, cols, vals)
    sense = (rng.random(m) < 0.30).astype(np.int8)
    l, u = _bounds_medium(rng, n)
    return construct(rng, m, n, rp, ci, v, sense, l, u, name=f"medium-{m}x{n}")


def _power_law_weights(k, exponent, total):
    # expected degree of the i-th node ~ i^(-1/(exponent-1)), scaled to sum to total
    w = np.arange(1, k + 1, dtype=np.float64) ** (-1.0 / (exponent - 1.0))
    return w * (total / w.sum())


def large(seed=SEED_BASE + 3, m=2_000_000, n=5_000_000, z=50_000_000, exponent=2.1,
          oversample=1.19) -> Problem:
    """2M x 5M, Chung-Lu power-law degrees, Z about 50M (see module docstring).

    Edges are drawn as oversample * z independent (row, column) pairs with
    P(row = i) and P(col = j) proportional to the power-law weights (the fast
    Chung-Lu sampler); repeated pairs are dropped (about 16% of the draws at
    these sizes, hence the oversampling), which also caps every row at n
    entries.  Node labels are shuffled so heavy rows/columns are not clustered."""
    rng = np.random.default_rng(seed)
    wr = _power_law_weights(m, exponent, z)
    wc = _power_law_weights(n, exponent, z)
    z = int(round(z * oversample))
    rperm = rng.permutation(m)
    cperm = rng.permutation(n)
    cr = np.cumsum(wr); cr /= cr[-1]
    cc = np.cumsum(wc); cc /= cc[-1]
    rows = rperm[np.minimum(np.searchsorted(cr, rng.random(z)), m - 1)]
    cols = cperm[np.minimum(np.searchsorted(cc, rng.random(z)), n - 1)]
    vals = rng.standard_normal(z)
    rp, ci, v = _csr_from_coo(m, rows, cols, vals)
    scale = np.exp(rng.normal(0.0, 3.0, m))
    v *= np.repeat(scale, np.diff(rp))
    sense = (rng.random(m) < 0.20).astype(np.int8)
    l, u = _bounds_medium(rng, n)
    return construct(rng, m, n, rp, ci, v, sense, l, u, name=f"large-{m}x{n}")


def banded(seed=SEED_BASE + 5, m=2_000_000, n=5_000_000, row_len=25) -> Problem:
    """m x n with row i holding the row_len consecutive columns starting at
    floor(i (n - row_len) / (m - 1)): every row has row_len entries and every
    column about row_len m / n (fewer at the two ends), so the degrees are
    nearly uniform and a longest-first renumbering keeps the columns of a
    degree class in order.  Values N(0,1) times a lognormal(0,3) scale per
    row, 20% '>=' rows, bounds as medium."""
    rng = np.random.default_rng(seed)
    start = (np.arange(m, dtype=np.int64) * (n - row_len)) // max(m - 1, 1)
    ci = (start[:, None] + np.arange(row_len, dtype=np.int64)[None, :]).astype(np.int32).ravel()
    rp = np.arange(m + 1, dtype=np.int64) * row_len
    v = rng.standard_normal(m * row_len) * np.repeat(np.exp(rng.normal(0.0, 3.0, m)), row_len)
    sense = (rng.random(m) < 0.20).astype(np.int8)
    l, u = _bounds_medium(rng, n)
    return construct(rng, m, n, rp, ci, v, sense, l, u, name=f"banded-{m}x{n}")


def batch_member(seed, m, n_per_m=2.5, nnz_mean=8.0, len_sigma=0.8) -> Problem:
    """One LP of the batched workload: m rows, round(n_per_m * m) columns, row
    lengths lognormal with mean nnz_mean (clipped to [1, min(2000, n)]) at
    uniform columns, N(0,1) values times a per-row lognormal(0, 2) scale, 30%
    '>=' rows, [0, U(1, 100)] bounds with 10% free variables; feasible with a
    known optimum by construction."""
    rng = np.random.default_rng(seed)
    n = int(round(n_per_m * m))
    mu = np.log(nnz_mean) - 0.5 * len_sigma ** 2
    lens = np.clip(np.rint(rng.lognormal(mu, len_sigma, m)).astype(np.int64), 1, min(2000, n))
    rows = np.repeat(np.arange(m, dtype=np.int64), lens)
    cols = rng.integers(0, n, len(rows))
    vals = rng.standard_normal(len(rows)) * np.exp(rng.normal(0.0, 2.0, m))[rows]
    rp, ci, v = _csr_from_coo(m, rows, cols, vals)
    sense = (rng.random(m) < 0.30).astype(np.int8)
    l, u = _bounds_medium(rng, n)
    return construct(rng, m, n, rp, ci, v, sense, l, u, name=f"batch-{m}x{n}")


def batch_sizes(seed=SEED_BASE + 4, count=256, rows_min=1_000, rows_max=50_000):
    """Row counts of the batched workload: log-uniform in [rows_min, rows_max]."""
    rng = np.random.default_rng(seed)
    return np.rint(np.exp(rng.uniform(np.log(rows_min), np.log(rows_max), count))).astype(np.int64)


def batch(seed=SEED_BASE + 4, count=256, rows_min=1_000, rows_max=50_000, scale=1.0):
    """The batched workload: `count` independent LPs of uneven size (rows
    log-uniform in [rows_min, rows_max], scaled by `scale`), member p drawn by
    batch_member with its own seed."""
    ms = batch_sizes(seed, count, rows_min, rows_max)
    return [batch_member(seed * 1000 + p, max(4, int(round(scale * int(mr))))) for p, mr in enumerate(ms)]


def toy_feasibility() -> Problem:
    """min 0 s.t. x = 3, x >= 0 (Sec. 5.2, eq. simple-feasibility); optimum
    (x, y) = (3, 0)."""
    P = Problem(1, 1, np.array([0, 1], np.int64), np.array([0], np.int32),
                np.array([1.0]), np.array([0], np.int8), np.array([3.0]), np.array([0.0]),
                np.array([0.0]), np.array([np.inf]), name="toy")
    P.x_star = np.array([3.0]); P.y_star = np.array([0.0]); P.lam_star = np.array([0.0])
    return P


def from_dense(Kd, sense, q, c, l, u, name="dense") -> Problem:
    """Problem from a dense matrix (tests only)."""
    Kd = np.asarray(Kd, dtype=np.float64)
    m, n = Kd.shape
    r, cidx = np.nonzero(Kd)
    rp = np.zeros(m + 1, np.int64)
    np.cumsum(np.bincount(r, minlength=m), out=rp[1:])
    return Problem(m, n, rp, cidx.astype(np.int32), Kd[r, cidx], np.asarray(sense, np.int8),
                   np.asarray(q, np.float64), np.asarray(c, np.float64),
                   np.asarray(l, np.float64), np.asarray(u, np.float64), name=name)


WORKLOADS = {"tiny": tiny, "medium": medium, "large": large, "banded": banded}
