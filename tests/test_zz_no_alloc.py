"""The allocation-free KKT entry point (aapdhg_kkt_noalloc), through the C ABI.

aapdhg_kkt_noalloc is for callers that cannot allocate device memory when they
need the residuals: loops that must not hit the implicit synchronisation of
cudaMalloc / cudaFree, and programs whose device memory is owned by another
framework's pool or a fixed budget.  It keeps its scratch in a fixed device
array, so this test checks two calls in a row (the second one must not see
the first one's leftovers) against the FP64 oracle's KKT and the existing
aapdhg_get_kkt, an LP without constraints (m = 0), and the rejection of sizes
beyond that array.  This file is collected last on purpose; it passes alone in
a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
from oracle import oracle as O

pytestmark = pytest.mark.gpu

RTOL = 1e-12      # same bar as the FP64 KKT parity test
KEYS = ("r_p", "r_d", "r_g", "kkt", "pobj", "dobj")


def _dev(t):
    return C.c_void_p(t.data_ptr())


def _problem():
    P = lpgen.random_lp(700, 1500, nnz_per_row=9, frac_ge=0.5, frac_free=0.2,
                        frac_lower_only=0.1, frac_upper_only=0.1, row_scale_sigma=1.0, seed=31)
    rng = np.random.default_rng(5)
    x = np.clip(P.x_star + 0.1 * rng.standard_normal(P.n), P.l, P.u)
    y = P.y_star + 0.1 * rng.standard_normal(P.m)
    y[P.sense == 1] = np.maximum(y[P.sense == 1], 0)
    return P, x, y


def _box_problem():
    """min c'x over a box only (m = 0): K has no rows."""
    rng = np.random.default_rng(9)
    n = 3000
    l = np.where(rng.random(n) < 0.2, -np.inf, -rng.uniform(0, 5, n))
    u = np.where(rng.random(n) < 0.2, np.inf, rng.uniform(0, 5, n))
    c = rng.standard_normal(n)
    x = np.clip(rng.standard_normal(n), l, u)
    return lpgen.Problem(0, n, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0),
                         np.zeros(0, np.int8), np.zeros(0), c, l, u), x, np.zeros(0)


def _get_kkt(P, x, y):
    from paper_2508_08062_gb300 import Solver
    with Solver(P, precision="fp64") as s:
        s.set_steps(0.1, 0.1)
        s.set_start(x, y)
        return s.get_kkt()


def _device_args(P, x, y):
    import torch
    K = sp.csr_matrix((P.val, P.col_idx.astype(np.int64), P.row_ptr), shape=(P.m, P.n))
    KT = K.T.tocsr()
    KT.sort_indices()

    def d(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        # a zero-length array still gets a real device buffer (one element)
        return torch.as_tensor(a if a.size else np.zeros(1, dt)).cuda()
    return [d(P.row_ptr, np.int64), d(P.col_idx, np.int32), d(P.val, np.float64),
            d(KT.indptr, np.int64), d(KT.indices, np.int32), d(KT.data, np.float64),
            d(P.sense, np.int8), d(P.q, np.float64), d(P.c, np.float64), d(P.l, np.float64),
            d(P.u, np.float64), d(x, np.float64), d(y, np.float64)]


def _noalloc(L, P, args):
    import torch
    out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    from paper_2508_08062_gb300 import binding
    rc = L.aapdhg_kkt_noalloc(P.m, P.n, *[_dev(a) for a in args], _dev(out),
                              C.c_void_p(stream.cuda_stream))
    assert rc == binding.OK
    torch.cuda.synchronize()
    return dict(zip(KEYS, out.cpu().numpy().tolist()))


def _close(got, ref, tag):
    for k in KEYS:
        assert abs(got[k] - ref[k]) <= RTOL * (abs(ref[k]) + 1e-3 * (1 + abs(ref["pobj"]))), \
            (tag, k, got[k], ref[k])


def test_noalloc_kkt_matches_oracle_and_get_kkt_twice():
    from paper_2508_08062_gb300 import binding
    L = binding.load()
    P, x, y = _problem()
    want = O.kkt(O.OracleLP.from_problem(P), x, y)
    ref = _get_kkt(P, x, y)
    args = _device_args(P, x, y)
    for call in range(2):
        got = _noalloc(L, P, args)
        _close(got, want, ("oracle", call))
        _close(got, ref, ("get_kkt", call))


def test_noalloc_kkt_without_constraints():
    from paper_2508_08062_gb300 import binding
    L = binding.load()
    P, x, y = _box_problem()
    want = O.kkt(O.OracleLP.from_problem(P), x, y)
    args = _device_args(P, x, y)
    for call in range(2):
        _close(_noalloc(L, P, args), want, ("box", call))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2508_08062_gb300 import binding
    L = binding.load()
    rows = 512 * (16384 + 1)                  # one block more than the fixed scratch holds
    dummy = C.c_void_p(16)                    # never dereferenced: the size check comes first
    rc = L.aapdhg_kkt_noalloc(0, rows, *([dummy] * 15))
    assert rc == binding.ERR_INVALID
