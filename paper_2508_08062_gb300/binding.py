"""Thin ctypes binding of the C ABI in ``include/aapdhg.h``.

Argument marshalling only: every step of the solver runs in the CUDA library
``libaapdhg.so``.  PyTorch supplies the device memory (its caching allocator is
installed as the library's allocator) and the CUDA stream (the current torch
stream by default).  There is no CPU fallback: if the library is missing or no
GPU is present, construction raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libaapdhg.so")

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_NUMERIC, ERR_TIMEOUT, NOT_CONVERGED = range(7)
TASK_SHAPES = 5
STATUS_NAMES = {0: "OK", 1: "ERR_INVALID", 2: "ERR_OOM", 3: "ERR_CUDA", 4: "ERR_NUMERIC",
                5: "ERR_TIMEOUT", 6: "NOT_CONVERGED"}
ROW_EQ, ROW_GE = 0, 1
FP64, MIXED = 0, 1
PDHG, AA, FAA = 0, 1, 2
MEM_HOST, MEM_DEVICE = 0, 1
METHODS = {"pdhg": PDHG, "aa": AA, "faa": FAA}
PRECISIONS = {"fp64": FP64, "mixed": MIXED}

# every entry point declared in include/aapdhg.h
EXPORTS = ("aapdhg_set_allocator", "aapdhg_create", "aapdhg_set_steps", "aapdhg_estimate_norm",
           "aapdhg_set_method", "aapdhg_set_scaling", "aapdhg_set_start", "aapdhg_reset",
           "aapdhg_iterate", "aapdhg_set_time_limit",
           "aapdhg_get_iterate", "aapdhg_get_kkt", "aapdhg_get_counters", "aapdhg_set_trace",
           "aapdhg_get_trace", "aapdhg_get_memory", "aapdhg_state_size", "aapdhg_get_state",
           "aapdhg_set_state", "aapdhg_profile_kernels",
           "aapdhg_get_kernel_profile",
           "aapdhg_kkt_noalloc", "aapdhg_device_bytes", "aapdhg_last_error", "aapdhg_destroy",
           "aapdhg_autotune", "aapdhg_set_task_shape", "aapdhg_set_layout",
           "aapdhg_autotune_layout", "aapdhg_batch_autotune", "aapdhg_batch_set_layout",
           "aapdhg_batch_autotune_layout",
           "aapdhg_set_primal_weight",
           "aapdhg_batch_set_task_shape", "aapdhg_batch_set_tolerances", "aapdhg_batch_launch",
           "aapdhg_batch_poll", "aapdhg_server_create", "aapdhg_server_submit",
           "aapdhg_server_step", "aapdhg_server_set_primal_weight", "aapdhg_server_result",
           "aapdhg_server_device_bytes",
           "aapdhg_server_last_error", "aapdhg_server_destroy",
           "aapdhg_batch_create", "aapdhg_batch_set_steps", "aapdhg_batch_estimate_norms",
           "aapdhg_batch_set_method", "aapdhg_batch_set_scaling", "aapdhg_batch_set_primal_weight",
           "aapdhg_batch_set_start",
           "aapdhg_batch_reset", "aapdhg_batch_iterate", "aapdhg_batch_get_iterate",
           "aapdhg_batch_get_kkt", "aapdhg_batch_get_member", "aapdhg_batch_get_status", "aapdhg_batch_profile_kernels",
           "aapdhg_batch_get_kernel_profile", "aapdhg_batch_device_bytes",
           "aapdhg_batch_last_error", "aapdhg_batch_destroy")
NO_STATUS = ("aapdhg_last_error", "aapdhg_destroy", "aapdhg_batch_last_error",
             "aapdhg_batch_destroy", "aapdhg_server_last_error", "aapdhg_server_destroy")


class AAPDHGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_alloc_cb = None
_free_cb = None


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises when it is missing: no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = C.CDLL(path)
    vp, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    st = C.c_int
    L.aapdhg_set_allocator.argtypes = [vp, vp, vp]
    L.aapdhg_create.argtypes = [i32, i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, i32, i32, vp,
                                C.POINTER(vp)]
    L.aapdhg_set_steps.argtypes = [vp, f64, f64]
    L.aapdhg_estimate_norm.argtypes = [vp, i32, C.c_uint64, C.POINTER(f64)]
    L.aapdhg_set_method.argtypes = [vp, i32, i32, f64, f64, f64, f64, f64, f64, f64, i32, i32]
    L.aapdhg_set_scaling.argtypes = [vp, i32, i32]
    L.aapdhg_set_start.argtypes = [vp, vp, vp]
    L.aapdhg_reset.argtypes = [vp]
    L.aapdhg_iterate.argtypes = [vp, i64, f64, i32, C.POINTER(i64)]
    L.aapdhg_set_time_limit.argtypes = [vp, f64]
    L.aapdhg_get_iterate.argtypes = [vp, vp, vp]
    L.aapdhg_get_kkt.argtypes = [vp, vp]
    L.aapdhg_get_counters.argtypes = [vp, vp, vp, vp, vp]
    L.aapdhg_set_trace.argtypes = [vp, i64]
    L.aapdhg_get_trace.argtypes = [vp, C.POINTER(i64), vp, vp, vp, vp]
    L.aapdhg_get_memory.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.aapdhg_state_size.argtypes = [vp, C.POINTER(C.c_size_t)]
    L.aapdhg_get_state.argtypes = [vp, vp, C.c_size_t]
    L.aapdhg_set_state.argtypes = [vp, vp, C.c_size_t]
    L.aapdhg_profile_kernels.argtypes = [vp, i32]
    L.aapdhg_get_kernel_profile.argtypes = [vp, i32, C.POINTER(i64), C.POINTER(f64)]
    L.aapdhg_kkt_noalloc.argtypes = [i32, i32] + [vp] * 15
    L.aapdhg_device_bytes.argtypes = [vp, C.POINTER(i64)]
    L.aapdhg_last_error.argtypes = [vp]
    L.aapdhg_last_error.restype = C.c_char_p
    L.aapdhg_destroy.argtypes = [vp]
    L.aapdhg_destroy.restype = None
    L.aapdhg_autotune.argtypes = [vp, vp, vp, vp]
    L.aapdhg_set_primal_weight.argtypes = [vp, i64, f64, f64, i32, f64, f64, f64]
    L.aapdhg_set_task_shape.argtypes = [vp, i32, i32]
    L.aapdhg_set_layout.argtypes = [vp, vp]
    L.aapdhg_autotune_layout.argtypes = [vp, vp, vp]
    L.aapdhg_batch_autotune.argtypes = [vp, vp, vp, vp]
    L.aapdhg_batch_set_task_shape.argtypes = [vp, i32, i32]
    L.aapdhg_batch_set_layout.argtypes = [vp, vp]
    L.aapdhg_batch_autotune_layout.argtypes = [vp, vp, vp]
    L.aapdhg_batch_create.argtypes = [i32] + [vp] * 11 + [i32, vp, C.POINTER(vp)]
    L.aapdhg_batch_set_tolerances.argtypes = [vp, vp]
    L.aapdhg_batch_launch.argtypes = [vp, i64, f64, i32]
    L.aapdhg_batch_poll.argtypes = [vp, vp]
    L.aapdhg_server_create.argtypes = [i32, i32, i32, i32, i64, i64, C.POINTER(vp)]
    L.aapdhg_server_submit.argtypes = [vp, i32, i32, i64] + [vp] * 8 + [f64, C.POINTER(i64)]
    L.aapdhg_server_step.argtypes = [vp, vp, vp]
    L.aapdhg_server_set_primal_weight.argtypes = [vp, i64, f64, f64, i32, f64, f64, f64]
    L.aapdhg_server_result.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
    L.aapdhg_server_device_bytes.argtypes = [vp, C.POINTER(i64)]
    L.aapdhg_server_last_error.argtypes = [vp]
    L.aapdhg_server_last_error.restype = C.c_char_p
    L.aapdhg_server_destroy.argtypes = [vp]
    L.aapdhg_server_destroy.restype = None
    L.aapdhg_batch_set_steps.argtypes = [vp, vp, vp]
    L.aapdhg_batch_estimate_norms.argtypes = [vp, i32, C.c_uint64, vp]
    L.aapdhg_batch_set_method.argtypes = [vp, i32, i32, f64, f64, f64, f64, f64, f64, f64, i32,
                                          i32]
    L.aapdhg_batch_set_scaling.argtypes = [vp, i32, i32]
    L.aapdhg_batch_set_primal_weight.argtypes = [vp, i64, f64, f64, i32, f64, f64, f64]
    L.aapdhg_batch_set_start.argtypes = [vp, vp, vp]
    L.aapdhg_batch_reset.argtypes = [vp]
    L.aapdhg_batch_iterate.argtypes = [vp, i64, f64, i32, C.POINTER(i64)]
    L.aapdhg_batch_get_iterate.argtypes = [vp, vp, vp]
    L.aapdhg_batch_get_kkt.argtypes = [vp, vp]
    L.aapdhg_batch_get_member.argtypes = [vp, i32, vp, vp, vp, vp]
    L.aapdhg_batch_get_status.argtypes = [vp, vp]
    L.aapdhg_batch_profile_kernels.argtypes = [vp, i32]
    L.aapdhg_batch_get_kernel_profile.argtypes = [vp, i32, C.POINTER(i64), C.POINTER(f64)]
    L.aapdhg_batch_device_bytes.argtypes = [vp, C.POINTER(i64)]
    L.aapdhg_batch_last_error.argtypes = [vp]
    L.aapdhg_batch_last_error.restype = C.c_char_p
    L.aapdhg_batch_destroy.argtypes = [vp]
    L.aapdhg_batch_destroy.restype = None
    for name in EXPORTS:
        if name not in NO_STATUS:
            getattr(L, name).restype = st
    _lib = L
    return L


def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator."""
    global _alloc_cb, _free_cb
    import torch
    L = load()
    ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
    FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

    def _alloc(nbytes, ctx):
        try:
            dev = torch.cuda.current_device()
            return torch.cuda.caching_allocator_alloc(int(nbytes), dev,
                                                      torch.cuda.current_stream(dev))
        except Exception:
            return None

    def _free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    _alloc_cb, _free_cb = ALLOC(_alloc), FREE(_free)
    L.aapdhg_set_allocator(C.cast(_alloc_cb, C.c_void_p), C.cast(_free_cb, C.c_void_p), None)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    assert a.shape == (n,), (a.shape, n)
    return a


class Solver:
    """One LP on the GPU (a handle of the C ABI).

    ``problem`` is any object with m, n, row_ptr, col_idx, val, sense, q, c, l, u
    (e.g. ``lpgen.Problem``).  ``device_inputs``: pass torch CUDA tensors as the
    attributes instead (int64 row_ptr, int32 col_idx, float64 values, int8 sense).
    """

    def __init__(self, problem, precision: str = "mixed", stream=None, torch_memory: bool = True,
                 device_inputs: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the solver has no CPU path")
        L = load()
        if torch_memory:
            use_torch_allocator()
        if stream is None:
            stream = torch.cuda.current_stream()
        self._L = L
        self._h = C.c_void_p()
        self.m, self.n = int(problem.m), int(problem.n)
        if device_inputs:
            def dp(t):
                return C.c_void_p(t.data_ptr())
            nnz = int(problem.val.numel())
            args = [dp(problem.row_ptr), dp(problem.col_idx), dp(problem.val), dp(problem.sense),
                    dp(problem.q), dp(problem.c), dp(problem.l), dp(problem.u)]
            kind = MEM_DEVICE
        else:
            rp = np.ascontiguousarray(problem.row_ptr, dtype=np.int64)
            ci = np.ascontiguousarray(problem.col_idx, dtype=np.int32)
            v = np.ascontiguousarray(problem.val, dtype=np.float64)
            se = np.ascontiguousarray(problem.sense, dtype=np.int8)
            self._keep = (rp, ci, v, se, _f64(problem.q, self.m), _f64(problem.c, self.n),
                          _f64(problem.l, self.n), _f64(problem.u, self.n))
            nnz = int(rp[-1])
            args = [_ptr(a) for a in self._keep]
            kind = MEM_HOST
        s = L.aapdhg_create(self.m, self.n, nnz, *args, PRECISIONS[precision], kind,
                            C.c_void_p(stream.cuda_stream), C.byref(self._h))
        if s != OK:
            raise AAPDHGError(s, L.aapdhg_last_error(None).decode())
        self._keep = None
        self.precision = precision

    # -- helpers -------------------------------------------------------------
    def _check(self, s, allow=(OK,)):
        if s not in allow:
            raise AAPDHGError(s, self._L.aapdhg_last_error(self._h).decode())
        return s

    def close(self):
        if self._h:
            self._L.aapdhg_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- C ABI ---------------------------------------------------------------
    def set_steps(self, tau, sigma):
        self._check(self._L.aapdhg_set_steps(self._h, float(tau), float(sigma)))

    def estimate_norm(self, iters=100, seed=1):
        out = C.c_double()
        self._check(self._L.aapdhg_estimate_norm(self._h, int(iters), int(seed), C.byref(out)))
        return out.value

    def set_method(self, method="aa", mem=5, D=10.0, eps=1.0, eta=1e-10, beta=1.0, c_s=0.2,
                   kappa=1e8, c_div=1.0, dhat_mode=1, faa_adaptive=1):
        m = METHODS[method] if isinstance(method, str) else int(method)
        self._check(self._L.aapdhg_set_method(self._h, m, int(mem), D, eps, eta, beta, c_s,
                                              kappa, c_div, int(dhat_mode), int(faa_adaptive)))

    def set_scaling(self, ruiz_iters=10, pock_chambolle=True):
        """Ruiz + Pock-Chambolle diagonal scaling (once per solver; resets the run)."""
        self._check(self._L.aapdhg_set_scaling(self._h, int(ruiz_iters), int(bool(pock_chambolle))))

    def set_primal_weight(self, period=3000, theta=0.5, eps_zero=1e-10, dhat_blend=True,
                          rho_min=0.1, alpha_dec=0.1, alpha_inc=0.9):
        """Periodic primal weight update (period 0: off); resets the run."""
        self._check(self._L.aapdhg_set_primal_weight(self._h, int(period), float(theta),
                                                     float(eps_zero), int(bool(dhat_blend)),
                                                     float(rho_min), float(alpha_dec),
                                                     float(alpha_inc)))

    def set_start(self, x0=None, y0=None):
        x0 = None if x0 is None else _f64(x0, self.n)
        y0 = None if y0 is None else _f64(y0, self.m)
        self._check(self._L.aapdhg_set_start(self._h, _ptr(x0), _ptr(y0)))

    def reset(self):
        self._check(self._L.aapdhg_reset(self._h))

    def iterate(self, max_iters, tol=0.0, kkt_every=0):
        """Returns (converged, iterations run).  Raises AAPDHGError on an error,
        including AAPDHG_ERR_TIMEOUT when the time limit ran out (not sticky)."""
        done = C.c_int64()
        s = self._L.aapdhg_iterate(self._h, int(max_iters), float(tol), int(kkt_every),
                                   C.byref(done))
        if s == ERR_TIMEOUT:
            err = AAPDHGError(s, "time limit ran out")
            err.iters_done = done.value
            raise err
        self._check(s, allow=(OK, NOT_CONVERGED))
        return s == OK, done.value

    def set_time_limit(self, seconds):
        """Wall-clock limit of the run in seconds (0: none)."""
        self._check(self._L.aapdhg_set_time_limit(self._h, float(seconds)))

    def get_iterate(self):
        x = np.empty(self.n)
        y = np.empty(self.m)
        self._check(self._L.aapdhg_get_iterate(self._h, _ptr(x), _ptr(y)))
        return x, y

    def get_kkt(self):
        out = np.empty(6)
        self._check(self._L.aapdhg_get_kkt(self._h, _ptr(out)))
        return dict(zip(("r_p", "r_d", "r_g", "kkt", "pobj", "dobj"), out.tolist()))

    def counters(self):
        v = np.zeros(4, dtype=np.int64)
        p = [C.c_void_p(v.ctypes.data + 8 * k) for k in range(4)]
        self._check(self._L.aapdhg_get_counters(self._h, *p))
        return dict(aa_steps=int(v[0]), pdhg_steps=int(v[1]), iters=int(v[2]),
                    ls_failures=int(v[3]))

    def set_trace(self, capacity):
        self._check(self._L.aapdhg_set_trace(self._h, int(capacity)))
        self._trace_cap = int(capacity)

    def get_trace(self):
        cap = getattr(self, "_trace_cap", 0)
        n = C.c_int64(cap)
        br = np.full(cap, -1, np.int8)
        gn = np.full(cap, np.nan)
        kk = np.full(cap, np.nan)
        mk = np.full(cap, -1, np.int32)
        self._check(self._L.aapdhg_get_trace(self._h, C.byref(n), _ptr(br), _ptr(gn), _ptr(kk),
                                             _ptr(mk)))
        k = n.value
        return dict(branch=br[:k], gnorm=gn[:k], kkt=kk[:k], mk=mk[:k])

    def autotune(self):
        """Time every task shape of the two half-step kernels now; returns the
        chosen shapes and the average launch time (us) of each shape."""
        sx, sy = C.c_int32(), C.c_int32()
        us = np.zeros(2 * TASK_SHAPES)
        self._check(self._L.aapdhg_autotune(self._h, C.byref(sx), C.byref(sy), _ptr(us)))
        return dict(shape_x=sx.value, shape_y=sy.value, x_us=us[:TASK_SHAPES].tolist(),
                    y_us=us[TASK_SHAPES:].tolist())

    def set_task_shape(self, shape_x, shape_y):
        """Fix the half-step task shapes ((-1, -1): tune again at the next iterate)."""
        self._check(self._L.aapdhg_set_task_shape(self._h, int(shape_x), int(shape_y)))

    def get_memory(self, capacity=32):
        """The Anderson memory after the last iteration (test hook): Gram matrix and
        right-hand side (oldest column first), the dG columns (count, n + m) and g^k."""
        cnt = C.c_int32()
        N = self.n + self.m
        gram = np.zeros(capacity * capacity); rhs = np.zeros(capacity)
        dg = np.zeros((capacity, N)); g = np.zeros(N)
        self._check(self._L.aapdhg_get_memory(self._h, int(capacity), C.byref(cnt), _ptr(gram),
                                               _ptr(rhs), _ptr(dg), _ptr(g)))
        k = cnt.value
        return dict(count=k, gram=gram[:k * k].reshape(k, k), rhs=rhs[:k], dg=dg[:k], g=g)

    def get_state(self):
        """The run's state blob (bytes): restoring it with set_state, here or in a
        handle made from the same LP with the same set-up, resumes the run exactly."""
        n = C.c_size_t()
        self._check(self._L.aapdhg_state_size(self._h, C.byref(n)))
        buf = np.zeros(n.value, dtype=np.uint8)
        self._check(self._L.aapdhg_get_state(self._h, _ptr(buf), n))
        return buf.tobytes()

    def set_state(self, blob):
        buf = np.frombuffer(bytes(blob), dtype=np.uint8).copy()
        self._check(self._L.aapdhg_set_state(self._h, _ptr(buf), C.c_size_t(buf.size)))

    LAYOUT_CANDIDATES = ((32, 1024), (16, 1024), (64, 1024), (128, 1024), (32, 2048), (64, 2048),
                         (128, 2048), (64, 4096))

    def set_layout(self, sell_max=32, long_chunk=1024, sell_max_y=None, long_chunk_y=None):
        """Rebuild the half-steps' matrix layouts: rows up to sell_max entries in
        SELL-32 slices, longer rows in chunks of long_chunk entries; the first
        pair for K' (x-step), the second (default: the same) for K (y-step)."""
        lay = np.array([sell_max, long_chunk, sell_max if sell_max_y is None else sell_max_y,
                        long_chunk if long_chunk_y is None else long_chunk_y], dtype=np.int32)
        self._check(self._L.aapdhg_set_layout(self._h, _ptr(lay)))

    def autotune_layout(self):
        """Time every candidate layout (with its task shapes tuned) and keep the
        fastest for each matrix; returns the choice and each candidate's best
        x / y launch (us)."""
        lay = np.zeros(4, dtype=np.int32)
        us = np.zeros(2 * len(self.LAYOUT_CANDIDATES))
        self._check(self._L.aapdhg_autotune_layout(self._h, _ptr(lay), _ptr(us)))
        return dict(x=(int(lay[0]), int(lay[1])), y=(int(lay[2]), int(lay[3])),
                    candidates=[dict(sell_max=a, long_chunk=b, x_us=us[2 * i], y_us=us[2 * i + 1])
                                for i, (a, b) in enumerate(self.LAYOUT_CANDIDATES)])

    KERNEL_KINDS = ("xstep", "ystep", "memory", "mix", "gram")

    def profile_kernels(self, enable=True):
        """CUDA-event timing of every kernel launched by iterate (resets totals)."""
        self._check(self._L.aapdhg_profile_kernels(self._h, int(bool(enable))))

    def kernel_profile(self):
        out = {}
        for k, name in enumerate(self.KERNEL_KINDS):
            n, ms = C.c_int64(), C.c_double()
            self._check(self._L.aapdhg_get_kernel_profile(self._h, k, C.byref(n), C.byref(ms)))
            out[name] = dict(launches=n.value, total_ms=ms.value,
                             avg_ms=(ms.value / n.value) if n.value else None)
        return out

    def launch_count(self):
        n, ms = C.c_int64(), C.c_double()
        self._check(self._L.aapdhg_get_kernel_profile(self._h, -1, C.byref(n), C.byref(ms)))
        return n.value

    def device_bytes(self):
        b = C.c_int64()
        self._check(self._L.aapdhg_device_bytes(self._h, C.byref(b)))
        return b.value


class BatchSolver:
    """Many independent LPs advanced together on the GPU (the batched C ABI).

    ``problems``: a sequence of objects like the ``Solver`` input.  Per-problem
    quantities go in and come out as arrays over the problems (step sizes,
    norms, KKT rows, status rows) or as lists of per-problem (x, y).
    """

    KERNEL_KINDS = ("xstep", "ystep", "memory", "mix", "kkt", "gram")

    def autotune(self):
        sx, sy = C.c_int32(), C.c_int32()
        us = np.zeros(2 * TASK_SHAPES)
        self._check(self._L.aapdhg_batch_autotune(self._h, C.byref(sx), C.byref(sy), _ptr(us)))
        return dict(shape_x=sx.value, shape_y=sy.value, x_us=us[:TASK_SHAPES].tolist(),
                    y_us=us[TASK_SHAPES:].tolist())

    def set_task_shape(self, shape_x, shape_y):
        self._check(self._L.aapdhg_batch_set_task_shape(self._h, int(shape_x), int(shape_y)))

    LAYOUT_CANDIDATES = Solver.LAYOUT_CANDIDATES

    def set_layout(self, sell_max=32, long_chunk=1024, sell_max_y=None, long_chunk_y=None):
        """As Solver.set_layout, on the packed K' and K."""
        lay = np.array([sell_max, long_chunk, sell_max if sell_max_y is None else sell_max_y,
                        long_chunk if long_chunk_y is None else long_chunk_y], dtype=np.int32)
        self._check(self._L.aapdhg_batch_set_layout(self._h, _ptr(lay)))

    def autotune_layout(self):
        """As Solver.autotune_layout, on the packed K' and K."""
        lay = np.zeros(4, dtype=np.int32)
        us = np.zeros(2 * len(self.LAYOUT_CANDIDATES))
        self._check(self._L.aapdhg_batch_autotune_layout(self._h, _ptr(lay), _ptr(us)))
        return dict(x=(int(lay[0]), int(lay[1])), y=(int(lay[2]), int(lay[3])),
                    candidates=[dict(sell_max=a, long_chunk=b, x_us=us[2 * i], y_us=us[2 * i + 1])
                                for i, (a, b) in enumerate(self.LAYOUT_CANDIDATES)])

    def __init__(self, problems, precision: str = "mixed", stream=None, torch_memory: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the solver has no CPU path")
        L = load()
        if torch_memory:
            use_torch_allocator()
        if stream is None:
            stream = torch.cuda.current_stream()
        self._L = L
        self._h = C.c_void_p()
        self.nprob = len(problems)
        self.m = np.array([int(P.m) for P in problems], dtype=np.int32)
        self.n = np.array([int(P.n) for P in problems], dtype=np.int32)
        nnz = np.array([int(np.asarray(P.row_ptr)[-1]) for P in problems], dtype=np.int64)
        cat = lambda key, dt: np.ascontiguousarray(  # noqa: E731
            np.concatenate([np.asarray(getattr(P, key), dtype=dt) for P in problems]), dtype=dt)
        keep = (self.m, self.n, nnz, cat("row_ptr", np.int64), cat("col_idx", np.int32),
                cat("val", np.float64), cat("sense", np.int8), cat("q", np.float64),
                cat("c", np.float64), cat("l", np.float64), cat("u", np.float64))
        s = L.aapdhg_batch_create(self.nprob, *[_ptr(a) for a in keep], PRECISIONS[precision],
                                  C.c_void_p(stream.cuda_stream), C.byref(self._h))
        if s != OK:
            raise AAPDHGError(s, L.aapdhg_batch_last_error(None).decode())
        self.xoff = np.concatenate([[0], np.cumsum(self.n.astype(np.int64))])
        self.yoff = np.concatenate([[0], np.cumsum(self.m.astype(np.int64))])
        self.precision = precision

    def _check(self, s, allow=(OK,)):
        if s not in allow:
            raise AAPDHGError(s, self._L.aapdhg_batch_last_error(self._h).decode())
        return s

    def close(self):
        if self._h:
            self._L.aapdhg_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_steps(self, tau, sigma):
        t = _f64(np.broadcast_to(np.asarray(tau, np.float64), (self.nprob,)), self.nprob)
        g = _f64(np.broadcast_to(np.asarray(sigma, np.float64), (self.nprob,)), self.nprob)
        self._check(self._L.aapdhg_batch_set_steps(self._h, _ptr(t), _ptr(g)))

    def estimate_norms(self, iters=100, seed=1):
        out = np.empty(self.nprob)
        self._check(self._L.aapdhg_batch_estimate_norms(self._h, int(iters), int(seed), _ptr(out)))
        return out

    def set_method(self, method="aa", mem=5, D=10.0, eps=1.0, eta=1e-10, beta=1.0, c_s=0.2,
                   kappa=1e8, c_div=1.0, dhat_mode=1, faa_adaptive=1):
        m = METHODS[method] if isinstance(method, str) else int(method)
        self._check(self._L.aapdhg_batch_set_method(self._h, m, int(mem), D, eps, eta, beta, c_s,
                                                    kappa, c_div, int(dhat_mode),
                                                    int(faa_adaptive)))

    def set_scaling(self, ruiz_iters=10, pock_chambolle=True):
        self._check(self._L.aapdhg_batch_set_scaling(self._h, int(ruiz_iters),
                                                     int(bool(pock_chambolle))))

    def set_primal_weight(self, period=3000, theta=0.5, eps_zero=1e-10, dhat_blend=True,
                          rho_min=0.1, alpha_dec=0.1, alpha_inc=0.9):
        """Periodic primal weight update of every problem on its own (period 0:
        off); resets the run."""
        self._check(self._L.aapdhg_batch_set_primal_weight(self._h, int(period), float(theta),
                                                           float(eps_zero), int(bool(dhat_blend)),
                                                           float(rho_min), float(alpha_dec),
                                                           float(alpha_inc)))

    def set_start(self, x0=None, y0=None):
        """x0, y0: concatenated caller-order arrays, or lists of per-problem arrays."""
        if isinstance(x0, (list, tuple)):
            x0 = np.concatenate(x0)
        if isinstance(y0, (list, tuple)):
            y0 = np.concatenate(y0) if len(y0) else np.zeros(0)
        x0 = None if x0 is None else _f64(x0, int(self.xoff[-1]))
        y0 = None if y0 is None else _f64(y0, int(self.yoff[-1]))
        self._check(self._L.aapdhg_batch_set_start(self._h, _ptr(x0), _ptr(y0)))

    def reset(self):
        self._check(self._L.aapdhg_batch_reset(self._h))

    def set_tolerances(self, tol):
        """Per-problem tolerances (None: one tolerance, the iterate argument, for all)."""
        t = None if tol is None else _f64(np.broadcast_to(np.asarray(tol, np.float64),
                                                          (self.nprob,)), self.nprob)
        self._check(self._L.aapdhg_batch_set_tolerances(self._h, _ptr(t)))

    def launch(self, n_iters, tol=0.0, kkt_every=0):
        """Enqueue n_iters batch iterations without waiting."""
        self._check(self._L.aapdhg_batch_launch(self._h, int(n_iters), float(tol), int(kkt_every)))

    def poll(self):
        """Wait for the enqueued work; True when every problem has stopped."""
        v = C.c_int32()
        self._check(self._L.aapdhg_batch_poll(self._h, C.byref(v)))
        return bool(v.value)

    def iterate(self, max_iters, tol=0.0, kkt_every=0):
        """Returns (all converged, batch iterations run)."""
        done = C.c_int64()
        s = self._check(self._L.aapdhg_batch_iterate(self._h, int(max_iters), float(tol),
                                                     int(kkt_every), C.byref(done)),
                        allow=(OK, NOT_CONVERGED, ERR_NUMERIC))
        return s == OK, done.value

    def get_iterate(self):
        x = np.empty(int(self.xoff[-1]))
        y = np.empty(int(self.yoff[-1]))
        self._check(self._L.aapdhg_batch_get_iterate(self._h, _ptr(x), _ptr(y)))
        return [(x[self.xoff[p]:self.xoff[p + 1]], y[self.yoff[p]:self.yoff[p + 1]])
                for p in range(self.nprob)]

    def get_kkt(self):
        """(nprob, 6) array: r_p, r_d, r_g, KKT, c'x, dual objective."""
        out = np.empty((self.nprob, 6))
        self._check(self._L.aapdhg_batch_get_kkt(self._h, _ptr(out)))
        return out

    def get_member(self, p):
        """One problem's (x, y), the KKT values of its last test and its status row."""
        p = int(p)
        x = np.empty(int(self.xoff[p + 1] - self.xoff[p]))
        y = np.empty(int(self.yoff[p + 1] - self.yoff[p]))
        kk = np.empty(6)
        st = np.empty(6, dtype=np.int64)
        self._check(self._L.aapdhg_batch_get_member(self._h, p, _ptr(x), _ptr(y), _ptr(kk), _ptr(st)))
        return x, y, kk, st

    def status(self):
        """(nprob, 6) int64: iterations, AA steps, PDHG steps, factorisation
        failures, converged, NaN/Inf met."""
        out = np.empty((self.nprob, 6), dtype=np.int64)
        self._check(self._L.aapdhg_batch_get_status(self._h, _ptr(out)))
        return out

    def profile_kernels(self, enable=True):
        self._check(self._L.aapdhg_batch_profile_kernels(self._h, int(bool(enable))))

    def kernel_profile(self):
        out = {}
        for k, name in enumerate(self.KERNEL_KINDS):
            n, ms = C.c_int64(), C.c_double()
            self._check(self._L.aapdhg_batch_get_kernel_profile(self._h, k, C.byref(n),
                                                                C.byref(ms)))
            out[name] = dict(launches=n.value, total_ms=ms.value,
                             avg_ms=(ms.value / n.value) if n.value else None)
        return out

    def launch_count(self):
        n, ms = C.c_int64(), C.c_double()
        self._check(self._L.aapdhg_batch_get_kernel_profile(self._h, -1, C.byref(n), C.byref(ms)))
        return n.value

    def device_bytes(self):
        b = C.c_int64()
        self._check(self._L.aapdhg_batch_device_bytes(self._h, C.byref(b)))
        return b.value


REQ_WAITING, REQ_RUNNING, REQ_CONVERGED, REQ_CAPPED, REQ_ERROR, REQ_REJECTED = range(6)
REQ_NAMES = ("waiting", "running", "converged", "capped", "error", "rejected")


class Server:
    """A served stream of LPs with continuous batching (the server C ABI)."""

    def __init__(self, method="aa", mem=10, max_cohorts=4, max_cohort_size=64, max_iters=100000,
                 mem_budget=0, torch_memory=True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the server has no CPU path")
        L = load()
        if torch_memory:
            use_torch_allocator()
        self._L = L
        self._h = C.c_void_p()
        m = METHODS[method] if isinstance(method, str) else int(method)
        s = L.aapdhg_server_create(m, int(mem), int(max_cohorts), int(max_cohort_size),
                                   int(max_iters), int(mem_budget), C.byref(self._h))
        if s != OK:
            raise AAPDHGError(s, L.aapdhg_server_last_error(None).decode())
        self._size = {}

    def _check(self, s):
        if s != OK:
            raise AAPDHGError(s, self._L.aapdhg_server_last_error(self._h).decode())

    def set_primal_weight(self, period=3000, theta=0.5, eps_zero=1e-10, dhat_blend=True,
                          rho_min=0.1, alpha_dec=0.1, alpha_inc=0.9):
        """Primal weight update for the cohorts admitted from now on (0: off)."""
        self._check(self._L.aapdhg_server_set_primal_weight(self._h, int(period), float(theta),
                                                            float(eps_zero), int(bool(dhat_blend)),
                                                            float(rho_min), float(alpha_dec),
                                                            float(alpha_inc)))

    def close(self):
        if self._h:
            self._L.aapdhg_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, P, tol):
        rp = np.ascontiguousarray(P.row_ptr, dtype=np.int64)
        arrs = (rp, np.ascontiguousarray(P.col_idx, dtype=np.int32),
                np.ascontiguousarray(P.val, dtype=np.float64),
                np.ascontiguousarray(P.sense, dtype=np.int8), _f64(P.q, P.m), _f64(P.c, P.n),
                _f64(P.l, P.n), _f64(P.u, P.n))
        rid = C.c_int64()
        self._check(self._L.aapdhg_server_submit(self._h, int(P.m), int(P.n), int(rp[-1]),
                                                 *[_ptr(a) for a in arrs], float(tol),
                                                 C.byref(rid)))
        self._size[rid.value] = (int(P.m), int(P.n))
        return rid.value

    def step(self):
        """One scheduling round; returns (cohorts running, LPs waiting)."""
        r, w = C.c_int32(), C.c_int32()
        self._check(self._L.aapdhg_server_step(self._h, C.byref(r), C.byref(w)))
        return r.value, w.value

    def result(self, rid):
        m, n = self._size[rid]
        st, it = C.c_int32(), C.c_int64(-1)
        x, y, kkt, t3 = np.full(n, np.nan), np.full(m, np.nan), np.full(6, np.nan), np.zeros(3)
        self._check(self._L.aapdhg_server_result(self._h, int(rid), C.byref(st), _ptr(x), _ptr(y),
                                                 _ptr(kkt), C.byref(it), _ptr(t3)))
        return dict(state=REQ_NAMES[st.value], x=x, y=y,
                    kkt=dict(zip(("r_p", "r_d", "r_g", "kkt", "pobj", "dobj"), kkt.tolist())),
                    iters=it.value, t_submit=t3[0], t_admit=t3[1], t_done=t3[2])

    def device_bytes(self):
        b = C.c_int64()
        self._check(self._L.aapdhg_server_device_bytes(self._h, C.byref(b)))
        return b.value
