"""Checkpoint / resume (aapdhg_get_state / aapdhg_set_state): a run restored
from its state blob continues bit for bit as the run it was taken from, on the
same handle and in a new handle made from the same LP with the same set-up;
blobs of another LP or set-up are refused."""
import numpy as np
import pytest

import lpgen

pytestmark = pytest.mark.gpu


def _solver(P, prec, mem=8, period=0, layout=None):
    from paper_2508_08062_gb300 import Solver
    s = Solver(P, precision=prec)
    s.set_scaling(10, True)
    nrm = s.estimate_norm(50, seed=1)
    s.set_steps(0.9 / nrm, 0.9 / nrm)
    s.set_method("aa", mem=mem, D=10.0, eps=1.0)
    if period:
        s.set_primal_weight(period=period)
    if layout:
        s.set_layout(*layout)
    return s


def _snapshot(s):
    x, y = s.get_iterate()
    return np.concatenate([x, y]), s.counters(), s.get_kkt()


@pytest.mark.parametrize("prec,period", [("fp64", 0), ("mixed", 0), ("mixed", 100), ("fp64", 100)])
def test_resume_is_exact(prec, period):
    P = lpgen.random_lp(3000, 7000, nnz_per_row=8, frac_ge=0.3, frac_free=0.1, seed=21)
    s = _solver(P, prec, period=period)
    s.iterate(130, tol=0.0, kkt_every=64)       # spans a primal weight update when period > 0
    blob = s.get_state()
    s.iterate(250, tol=0.0, kkt_every=64)
    u1, c1, k1 = _snapshot(s)
    assert c1["aa_steps"] > 0
    # the same handle, rewound
    s.set_state(blob)
    s.iterate(250, tol=0.0, kkt_every=64)
    u2, c2, k2 = _snapshot(s)
    assert np.array_equal(u1, u2)
    assert c1 == c2 and k1 == k2
    s.close()
    # a new handle, same LP and set-up, but another layout before the restore
    t = _solver(P, prec, period=period, layout=(16, 512))
    t.set_state(blob)
    t.iterate(250, tol=0.0, kkt_every=64)
    u3, c3, k3 = _snapshot(t)
    t.close()
    assert np.array_equal(u1, u3)
    assert c1 == c3
    # the KKT terms' block partials are summed over this handle's tuned grids
    for key in k1:
        assert k3[key] == pytest.approx(k1[key], rel=1e-12, abs=1e-300), key


def test_foreign_blobs_are_refused():
    from paper_2508_08062_gb300 import AAPDHGError
    P = lpgen.random_lp(300, 700, nnz_per_row=6, seed=5)
    Q = lpgen.random_lp(301, 700, nnz_per_row=6, seed=5)
    with _solver(P, "mixed") as s:
        s.iterate(20)
        blob = s.get_state()
    for make in (lambda: _solver(Q, "mixed"),               # another LP
                 lambda: _solver(P, "fp64"),                # another precision
                 lambda: _solver(P, "mixed", mem=5),        # another memory
                 lambda: _solver(P, "mixed", period=50)):   # another primal weight period
        with make() as t:
            with pytest.raises(AAPDHGError):
                t.set_state(blob)
    with _solver(P, "mixed") as t:
        with pytest.raises(AAPDHGError):
            t.set_state(blob[:-8])                           # truncated
    with _solver(P, "mixed") as t:
        bad = bytearray(blob)
        bad[0] ^= 0xFF                                       # not a blob of this library
        with pytest.raises(AAPDHGError):
            t.set_state(bytes(bad))
