"""ctypes binding of the FP64 CPU oracle (``aapdhg_oracle.c``).

Test infrastructure: only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this module.  It converts numpy arrays to
pointers and nothing else; every formula lives in the C file, which cites the
paper's sections, equations and algorithms.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aapdhg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no FMA contraction so that x86 and
    Arm hosts round identically)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _LP(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("rp", C.c_void_p), ("ci", C.c_void_p),
                ("v", C.c_void_p), ("sense", C.c_void_p), ("q", C.c_void_p), ("c", C.c_void_p),
                ("l", C.c_void_p), ("u", C.c_void_p)]


class _Params(C.Structure):
    _fields_ = [("method", C.c_int32), ("mem", C.c_int32), ("tau", C.c_double),
                ("sigma", C.c_double), ("D", C.c_double), ("eps", C.c_double),
                ("eta", C.c_double), ("beta", C.c_double), ("c_s", C.c_double),
                ("kappa", C.c_double), ("c_div", C.c_double), ("dhat_mode", C.c_int32),
                ("faa_adaptive", C.c_int32), ("pw_period", C.c_int32), ("pw_theta", C.c_double),
                ("pw_eps_zero", C.c_double), ("pw_dhat", C.c_int32), ("pw_rho_min", C.c_double),
                ("pw_alpha_dec", C.c_double), ("pw_alpha_inc", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        vp = C.c_void_p
        L.orc_dhat.argtypes = [vp, C.c_int32, vp, vp]
        L.orc_T.argtypes = [vp, C.c_double, C.c_double, vp, vp, vp, vp]
        L.orc_kkt.argtypes = [vp, vp, vp, vp]
        L.orc_aa_coeffs.argtypes = [C.c_int64, C.c_int32, vp, vp, C.c_double, vp]
        L.orc_aa_coeffs.restype = C.c_int
        L.orc_aa_mix.argtypes = [C.c_int64, C.c_int32, vp, vp, vp, vp, vp, C.c_double, vp, vp]
        L.orc_qr_coeffs.argtypes = [C.c_int64, C.c_int32, vp, vp, vp]
        L.orc_qr_coeffs.restype = C.c_int
        L.orc_length_bounds.argtypes = [C.c_int32, vp, C.c_double, vp]
        L.orc_faa_filter.argtypes = [C.c_int64, C.c_int32, vp, vp, C.c_double, C.c_double, vp]
        L.orc_faa_filter.restype = C.c_int32
        L.orc_solve.argtypes = [vp, vp, vp, vp, C.c_int64, C.c_double, C.c_int32, vp, vp, vp,
                                C.c_int64, vp, vp, vp, vp, C.c_int64, vp, vp]
        L.orc_solve.restype = C.c_int
        L.orc_scaling.argtypes = [vp, C.c_int32, C.c_int32, vp, vp]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


class OracleLP:
    """The LP of eq. LP-O in the oracle's layout: K = [G; A] as FP64 CSR with
    int64 row pointers, a sense byte per row (1: '>=', 0: '=')."""

    def __init__(self, m, n, row_ptr, col_idx, val, sense, q, c, l, u):
        self.m, self.n = int(m), int(n)
        self.rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        self.v = np.ascontiguousarray(val, dtype=np.float64)
        self.sense = np.ascontiguousarray(sense, dtype=np.int8)
        self.q = np.ascontiguousarray(q, dtype=np.float64)
        self.c = np.ascontiguousarray(c, dtype=np.float64)
        self.l = np.ascontiguousarray(l, dtype=np.float64)
        self.u = np.ascontiguousarray(u, dtype=np.float64)
        assert self.rp.shape == (self.m + 1,) and self.q.shape == (self.m,)
        assert self.c.shape == (self.n,) and self.sense.shape == (self.m,)
        self._s = _LP(self.m, self.n, _p(self.rp), _p(self.ci), _p(self.v), _p(self.sense),
                      _p(self.q), _p(self.c), _p(self.l), _p(self.u))

    @classmethod
    def from_problem(cls, P):
        return cls(P.m, P.n, P.row_ptr, P.col_idx, P.val, P.sense, P.q, P.c, P.l, P.u)

    @property
    def ref(self):
        return C.byref(self._s)


@dataclass
class Params:
    method: int = 1          # 0 PDHG, 1 AA-PDHG, 2 FAA-PDHG
    mem: int = 5
    tau: float = 0.1
    sigma: float = 0.1
    D: float = 10.0
    eps: float = 1.0
    eta: float = 1e-10
    beta: float = 1.0
    c_s: float = 0.2
    kappa: float = 1e8
    c_div: float = 1.0
    dhat_mode: int = 1
    faa_adaptive: int = 1
    pw_period: int = 0       # primal weight update every pw_period iterations (0: off)
    pw_theta: float = 0.5
    pw_eps_zero: float = 1e-10
    pw_dhat: int = 1
    pw_rho_min: float = 0.1
    pw_alpha_dec: float = 0.1
    pw_alpha_inc: float = 0.9

    def _struct(self):
        return _Params(self.method, self.mem, self.tau, self.sigma, self.D, self.eps, self.eta,
                       self.beta, self.c_s, self.kappa, self.c_div, self.dhat_mode,
                       self.faa_adaptive, self.pw_period, self.pw_theta, self.pw_eps_zero,
                       self.pw_dhat, self.pw_rho_min, self.pw_alpha_dec, self.pw_alpha_inc)


def dhat(lp: OracleLP, mode: int = 1):
    dx = np.empty(lp.n); dy = np.empty(lp.m)
    lib().orc_dhat(lp.ref, mode, _p(dx), _p(dy))
    return dx, dy


def scaling(lp: OracleLP, ruiz_iters: int = 10, pock_chambolle: bool = True):
    """Row and column factors (dr, dc) of the preconditioning (reading R12)."""
    dr = np.empty(lp.m); dc = np.empty(lp.n)
    lib().orc_scaling(lp.ref, int(ruiz_iters), int(bool(pock_chambolle)), _p(dr), _p(dc))
    return dr, dc


def scaled_lp(lp: OracleLP, dr, dc) -> OracleLP:
    """The scaled LP: Dr K Dc, Dr q, Dc c, bounds / Dc (x = Dc x~, y = Dr y~)."""
    rows = np.repeat(np.arange(lp.m), np.diff(lp.rp))
    return OracleLP(lp.m, lp.n, lp.rp, lp.ci, dr[rows] * lp.v * dc[lp.ci], lp.sense, dr * lp.q,
                    dc * lp.c, lp.l / dc, lp.u / dc)


def T(lp: OracleLP, tau, sigma, x, y):
    x = np.ascontiguousarray(x, dtype=np.float64); y = np.ascontiguousarray(y, dtype=np.float64)
    xh = np.empty(lp.n); yh = np.empty(lp.m)
    lib().orc_T(lp.ref, tau, sigma, _p(x), _p(y), _p(xh), _p(yh))
    return xh, yh


def kkt(lp: OracleLP, x, y):
    """Returns dict with r_p, r_d, r_g, kkt, pobj, dobj."""
    x = np.ascontiguousarray(x, dtype=np.float64); y = np.ascontiguousarray(y, dtype=np.float64)
    out = np.empty(6)
    lib().orc_kkt(lp.ref, _p(x), _p(y), _p(out))
    return dict(zip(("r_p", "r_d", "r_g", "kkt", "pobj", "dobj"), out.tolist()))


def aa_coeffs(dG, g, eta):
    """gamma = (dG'dG + eta I)^-1 dG'g; dG is (N, k).  Returns (rc, gamma)."""
    N, k = dG.shape
    F = np.ascontiguousarray(dG.T, dtype=np.float64)    # column-major columns
    g = np.ascontiguousarray(g, dtype=np.float64)
    gam = np.zeros(k)
    rc = lib().orc_aa_coeffs(N, k, _p(F), _p(g), eta, _p(gam))
    return rc, gam


def aa_mix(u, g, dU, dG, dhat, beta, gamma):
    """u + beta D-hat g - (dU + beta D-hat dG) gamma (the AA step of Alg. 2
    before the projection); dU, dG are (N, k)."""
    N, k = dG.shape
    E = np.ascontiguousarray(dU.T, dtype=np.float64)
    F = np.ascontiguousarray(dG.T, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64); g = np.ascontiguousarray(g, dtype=np.float64)
    dh = np.ascontiguousarray(dhat, dtype=np.float64)
    gam = np.ascontiguousarray(gamma, dtype=np.float64)
    out = np.empty(N)
    lib().orc_aa_mix(N, k, _p(u), _p(g), _p(E), _p(F), _p(dh), float(beta), _p(gam), _p(out))
    return out


def qr_coeffs(dG, g):
    N, k = dG.shape
    F = np.ascontiguousarray(dG.T, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    gam = np.zeros(k)
    rc = lib().orc_qr_coeffs(N, k, _p(F), _p(g), _p(gam))
    return rc, gam


def length_bounds(fnorms, c_s):
    fn = np.ascontiguousarray(fnorms, dtype=np.float64)
    b = np.empty(len(fn))
    lib().orc_length_bounds(len(fn), _p(fn), c_s, _p(b))
    return b


def faa_filter(dU, dG, c_s, kappa):
    """Kept-column mask (oldest-first indexing) of Reverse/AngleFilter/LengthFilter/Reverse."""
    N, k = dG.shape
    E = np.ascontiguousarray(dU.T, dtype=np.float64)
    F = np.ascontiguousarray(dG.T, dtype=np.float64)
    keep = np.zeros(k, dtype=np.int32)
    lib().orc_faa_filter(N, k, _p(E), _p(F), c_s, kappa, _p(keep))
    return keep.astype(bool)


@dataclass
class SolveResult:
    status: int              # 0 converged (KKT <= tol), 1 iteration cap
    x: np.ndarray
    y: np.ndarray
    aa_steps: int
    pdhg_steps: int
    iters: int
    branch: np.ndarray | None = None
    gnorm: np.ndarray | None = None
    kkt: np.ndarray | None = None
    mk: np.ndarray | None = None
    rec_u: np.ndarray | None = None
    dhat: np.ndarray | None = None       # D-hat in use at the end (primal weight re-blend)


def solve(lp: OracleLP, params: Params, max_iters: int, tol: float = 0.0, kkt_every: int = 0,
          x0=None, y0=None, trace: bool = False, rec_len: int = 0) -> SolveResult:
    x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    y0 = None if y0 is None else np.ascontiguousarray(y0, dtype=np.float64)
    x = np.empty(lp.n); y = np.empty(lp.m)
    counters = np.zeros(3, dtype=np.int64)
    tl = max_iters if trace else 0
    br = np.full(tl, -1, dtype=np.int8) if trace else None
    gn = np.full(tl, np.nan) if trace else None
    kk = np.full(tl, np.nan) if trace else None
    mk = np.full(tl, -1, dtype=np.int32) if trace else None
    rec = np.full((rec_len, lp.n + lp.m), np.nan) if rec_len > 0 else None
    ps = params._struct()
    dh = np.empty(lp.n + lp.m)
    rc = lib().orc_solve(lp.ref, C.byref(ps), _p(x0), _p(y0), max_iters, tol, kkt_every, _p(x),
                         _p(y), _p(counters), tl, _p(br), _p(gn), _p(kk), _p(mk), rec_len, _p(rec),
                         _p(dh))
    it = int(counters[2])
    res = SolveResult(rc, x, y, int(counters[0]), int(counters[1]), it)
    res.dhat = dh
    if trace:
        res.branch, res.gnorm, res.kkt, res.mk = br[:it + 1], gn[:it + 1], kk[:it + 1], mk[:it + 1]
    if rec is not None:
        res.rec_u = rec[:min(rec_len, it + 1)]
    return res
