"""The allocation-free KKT entry point (aapdhg_kkt_noalloc) against the existing
aapdhg_get_kkt, through the C ABI.

aapdhg_kkt_noalloc is for callers that cannot allocate device memory when they
need the residuals (during stream capture, in loops that must not hit the
implicit synchronisation of cudaMalloc / cudaFree, or when another framework
owns the device memory).  It keeps its scratch in a fixed device array, so this
test checks two calls in a row (the second one must not see the first one's
leftovers) and the rejection of sizes beyond that array.  This file is
collected last on purpose; it passes alone in a fresh process as well.
"""
import ctypes as C

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen

pytestmark = pytest.mark.gpu

RTOL = 1e-12      # same bar as the FP64 KKT parity test


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


def _reference(P, x, y):
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
    d = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a, dtype=dt)).cuda()
    return [d(P.row_ptr, np.int64), d(P.col_idx, np.int32), d(P.val, np.float64),
            d(KT.indptr, np.int64), d(KT.indices, np.int32), d(KT.data, np.float64),
            d(P.sense, np.int8), d(P.q, np.float64), d(P.c, np.float64), d(P.l, np.float64),
            d(P.u, np.float64), d(x, np.float64), d(y, np.float64)]


def test_noalloc_kkt_matches_get_kkt_twice():
    import torch
    from paper_2508_08062_gb300 import binding
    L = binding.load()
    P, x, y = _problem()
    ref = _reference(P, x, y)
    args = _device_args(P, x, y)
    keys = ("r_p", "r_d", "r_g", "kkt", "pobj", "dobj")
    stream = torch.cuda.current_stream()
    for call in range(2):
        out = torch.full((6,), float("nan"), dtype=torch.float64, device="cuda")
        rc = L.aapdhg_kkt_noalloc(P.m, P.n, *[_dev(a) for a in args], _dev(out),
                                  C.c_void_p(stream.cuda_stream))
        assert rc == binding.OK
        torch.cuda.synchronize()
        got = dict(zip(keys, out.cpu().numpy().tolist()))
        for k in keys:
            assert abs(got[k] - ref[k]) <= RTOL * (abs(ref[k]) + 1e-3 * (1 + abs(ref["pobj"]))), \
                (call, k, got[k], ref[k])


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2508_08062_gb300 import binding
    L = binding.load()
    rows = 512 * (16384 + 1)                  # one block more than the fixed scratch holds
    dummy = C.c_void_p(16)                    # never dereferenced: the size check comes first
    rc = L.aapdhg_kkt_noalloc(0, rows, *([dummy] * 15))
    assert rc == binding.ERR_INVALID
