"""Input validation of the C ABI's create calls, on the CPU.

aapdhg_create and aapdhg_batch_create check their input before any CUDA
call, so a malformed LP is refused here, with the message of the first
failing check: rows in order (a row's sense, then its columns), then the
values, then the bounds; for a batch, the lowest failing problem.  The LPs
are large enough (> 2^20 nonzeros) for the checks to run on several threads,
whose verdicts must match that order.
"""
import ctypes as C

import numpy as np

from paper_2508_08062_gb300 import binding

M, N, W = 140_000, 300_000, 8          # rows, columns, entries per row (1.12M nonzeros)


def _lp(m=M, n=N, w=W):
    rp = np.arange(0, w * (m + 1), w, dtype=np.int64)
    ci = ((np.arange(m, dtype=np.int64)[:, None] * 5 + np.arange(w)[None, :] * 7) % n).astype(np.int32).ravel()
    return dict(m=m, n=n, rp=rp, ci=ci, val=np.ones(m * w), sense=np.zeros(m, np.int8), q=np.zeros(m),
                c=np.zeros(n), lb=np.zeros(n), ub=np.ones(n))


def _create(d):
    L = binding.load()
    h = C.c_void_p()
    s = L.aapdhg_create(d["m"], d["n"], len(d["ci"]), d["rp"].ctypes.data, d["ci"].ctypes.data,
                        d["val"].ctypes.data, d["sense"].ctypes.data, d["q"].ctypes.data, d["c"].ctypes.data,
                        d["lb"].ctypes.data, d["ub"].ctypes.data, binding.MIXED, binding.MEM_HOST, None,
                        C.byref(h))
    if s == binding.OK:                  # a machine with a GPU built it
        L.aapdhg_destroy(h)
    return s, L.aapdhg_last_error(None).decode()


def _expect(d, msg):
    s, err = _create(d)
    assert s == binding.ERR_INVALID and err == msg, (s, err)


def test_valid_input_passes_the_checks():
    s, err = _create(_lp())
    assert s != binding.ERR_INVALID, err


def test_the_first_failing_row_decides():
    d = _lp()
    d["ci"] = d["ci"].copy()
    d["ci"][W * 120_000 + 3] = N                      # column out of range, late row
    d["ci"][W * 9_000 + 5] = d["ci"][W * 9_000 + 2]   # repeated column, early row
    _expect(d, "repeated column within a row")
    d["sense"] = d["sense"].copy()
    d["sense"][100] = 7                              # an earlier row still: its sense
    _expect(d, "row_sense must be 0 (=) or 1 (>=)")


def test_row_pointers():
    d = _lp()
    d["rp"] = d["rp"].copy()
    d["rp"][70_000] = d["rp"][70_001] + 1            # decreases after row 70k
    _expect(d, "row_ptr is not non-decreasing")
    d["ci"] = d["ci"].copy()
    d["ci"][W * 10] = -1                             # a bad column before it comes first
    _expect(d, "column index out of range")
    e = _lp()
    e["rp"] = e["rp"].copy()
    e["rp"][50_000:50_003] = 10 * len(e["ci"])       # beyond nnz, then back: refused, not read
    _expect(e, "row_ptr is not non-decreasing")
    f = _lp()
    f["rp"] = f["rp"].copy()
    f["rp"][-1] += 1
    _expect(f, "row_ptr[0] must be 0 and row_ptr[m] must be nnz")


def test_values_then_bounds():
    d = _lp()
    d["val"] = d["val"].copy()
    d["val"][-5] = np.inf
    d["lb"] = d["lb"].copy()
    d["lb"][3] = 2.0                                 # lb > ub as well: the values come first
    _expect(d, "non-finite value in K, q or c")
    d["val"][-5] = 1.0
    _expect(d, "bounds must satisfy lb <= ub, lb < +inf, ub > -inf")
    d["lb"][3] = 0.0
    d["q"] = d["q"].copy()
    d["q"][M - 1] = np.nan
    _expect(d, "non-finite value in K, q or c")


def test_batch_reports_the_lowest_failing_problem():
    L = binding.load()
    probs = [_lp(m=30_000, n=60_000) for _ in range(6)]   # 1.44M nonzeros in all
    probs[4]["sense"] = probs[4]["sense"].copy()
    probs[4]["sense"][7] = 3
    probs[2]["ci"] = probs[2]["ci"].copy()
    probs[2]["ci"][W * 29_000] = 60_000
    cat = lambda k, t: np.ascontiguousarray(np.concatenate([p[k] for p in probs]).astype(t))
    m = np.array([p["m"] for p in probs], np.int32)
    n = np.array([p["n"] for p in probs], np.int32)
    nnz = np.array([len(p["ci"]) for p in probs], np.int64)
    arrs = [cat("rp", np.int64), cat("ci", np.int32), cat("val", np.float64), cat("sense", np.int8),
            cat("q", np.float64), cat("c", np.float64), cat("lb", np.float64), cat("ub", np.float64)]
    h = C.c_void_p()
    s = L.aapdhg_batch_create(len(probs), m.ctypes.data, n.ctypes.data, nnz.ctypes.data,
                              *[a.ctypes.data for a in arrs], binding.MIXED, None, C.byref(h))
    assert s == binding.ERR_INVALID
    assert L.aapdhg_batch_last_error(None).decode() == "problem 2: column index out of range"


def test_kkt_noalloc_refuses_null_pointers():
    """aapdhg_kkt_noalloc checks its pointers before any CUDA call: a NULL for
    any array it reads gives AAPDHG_ERR_INVALID.  Its 14 array arguments come
    first (the 15th, the stream, may be NULL); with m > 0 every array is
    required.  Each call below has exactly one NULL array, so none of them
    reaches the device."""
    L = binding.load()
    dummy = C.c_void_p(16)                    # never dereferenced: the check comes first
    for i in range(14):
        args = [dummy] * 14 + [None]
        args[i] = None
        assert L.aapdhg_kkt_noalloc(10, 20, *args) == binding.ERR_INVALID, i
    # with m = 0 only K's row pointers, K' row pointers, c, lb, ub, x and out6 are read
    for i in (0, 3, 8, 9, 10, 11, 13):
        args = [dummy] * 14 + [None]
        args[i] = None
        assert L.aapdhg_kkt_noalloc(0, 20, *args) == binding.ERR_INVALID, i


def test_state_calls_refuse_a_null_handle():
    """The checkpoint calls check the handle before anything else."""
    L = binding.load()
    n = C.c_size_t(7)
    assert L.aapdhg_state_size(None, C.byref(n)) == binding.ERR_INVALID
    assert n.value == 7
    buf = (C.c_uint8 * 64)()
    assert L.aapdhg_get_state(None, buf, 64) == binding.ERR_INVALID
    assert L.aapdhg_set_state(None, buf, 64) == binding.ERR_INVALID
