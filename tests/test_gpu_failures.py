"""Failure statuses of the C ABI, produced on the host (no GPU fault is made).

* AAPDHG_ERR_OOM: a capped allocator, installed with aapdhg_set_allocator,
  refuses allocations beyond its budget: at create, and later for the trace
  buffers (sticky from then on).
* AAPDHG_ERR_NUMERIC: step sizes far beyond the stability bound of eq. pdhg
  make the iterate overflow; the device stops on the NaN/Inf and the host
  reports it (sticky for one LP; per problem, not sticky, in a batch).
* AAPDHG_ERR_TIMEOUT: the time limit of a run (the one-hour cap of the
  experiments, here a few milliseconds) runs out between chunks; the run stays
  resumable.
"""
import ctypes as C

import numpy as np
import pytest

import lpgen

pytestmark = pytest.mark.gpu


class _CappedAllocator:
    """torch's caching allocator behind a byte budget (NULL beyond it)."""

    def __init__(self, cap):
        import torch
        self.cap, self.used, self.sizes, self.refused = cap, 0, {}, 0
        ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
        FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

        def _alloc(nbytes, ctx):
            if self.used + nbytes > self.cap:
                self.refused += 1
                return None
            dev = torch.cuda.current_device()
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, torch.cuda.current_stream(dev))
            self.sizes[p] = int(nbytes)
            self.used += int(nbytes)
            return p

        def _free(ptr, ctx):
            self.used -= self.sizes.pop(ptr)
            torch.cuda.caching_allocator_delete(ptr)

        self._a, self._f = ALLOC(_alloc), FREE(_free)

    def install(self):
        from paper_2508_08062_gb300 import binding
        binding.load().aapdhg_set_allocator(C.cast(self._a, C.c_void_p), C.cast(self._f, C.c_void_p),
                                            None)


def test_out_of_memory_at_create_and_later():
    from paper_2508_08062_gb300 import AAPDHGError, Solver, binding
    P = lpgen.random_lp(2000, 5000, nnz_per_row=8, seed=3)
    cap = _CappedAllocator(64 * 1024)              # far below what the LP needs
    cap.install()
    try:
        with pytest.raises(AAPDHGError) as e:
            Solver(P, precision="mixed", torch_memory=False)
        assert e.value.status == binding.ERR_OOM
        assert "allocation" in str(e.value)
        assert cap.refused >= 1 and cap.used == 0    # what create got is returned
        cap.cap = 1 << 40
        with Solver(P, precision="mixed", torch_memory=False) as s:
            s.set_steps(0.1, 0.1)
            s.iterate(10)
            cap.cap = cap.used                     # nothing more fits
            with pytest.raises(AAPDHGError) as e:
                s.set_trace(1000)
            assert e.value.status == binding.ERR_OOM and "trace" in str(e.value)
            with pytest.raises(AAPDHGError) as e:  # sticky
                s.get_iterate()
            assert e.value.status == binding.ERR_OOM
        assert cap.used == 0                       # destroy returns everything
    finally:
        binding.use_torch_allocator()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_numeric_overflow_is_reported_and_sticky(prec):
    from paper_2508_08062_gb300 import AAPDHGError, Solver, binding
    P = lpgen.random_lp(300, 700, nnz_per_row=6, frac_ge=0.3, frac_free=0.5, seed=8)
    with Solver(P, precision=prec) as s:
        s.set_steps(1e150, 1e150)                  # sigma tau ||K||^2 >> 1
        s.set_method("aa", mem=5)
        with pytest.raises(AAPDHGError) as e:
            s.iterate(5000)
        assert e.value.status == binding.ERR_NUMERIC
        assert "NaN or Inf" in str(e.value)
        with pytest.raises(AAPDHGError) as e:
            s.get_kkt()
        assert e.value.status == binding.ERR_NUMERIC


def test_numeric_overflow_in_one_batch_member():
    """One LP of a batch overflows; it stops with its NaN/Inf flag and the
    others converge (the batch reports AAPDHG_ERR_NUMERIC, not sticky)."""
    from paper_2508_08062_gb300 import BatchSolver
    probs = [lpgen.random_lp(60, 120, nnz_per_row=5, frac_ge=0.3, frac_free=0.5, seed=s)
             for s in (3, 4, 5)]
    with BatchSolver(probs, precision="fp64") as b:
        nrm = b.estimate_norms(200, seed=1)
        taus = 0.9 / nrm
        taus[1] = 1e150
        b.set_steps(taus, taus)
        b.set_method("aa", mem=5)
        conv, _ = b.iterate(200000, tol=1e-4, kkt_every=16)
        st = b.status()
        assert not conv
        assert st[1, 5] == 1 and st[1, 4] == 0
        assert st[0, 4] == 1 and st[2, 4] == 1 and st[0, 5] == 0 and st[2, 5] == 0
        x, y = b.get_iterate()[0]                  # the handle stays usable
        assert np.all(np.isfinite(x))


def _tiny_steps(P):
    import scipy.sparse as sp
    K = sp.csr_matrix((P.val, P.col_idx.astype(np.int64), P.row_ptr), shape=(P.m, P.n))
    return 0.9 / np.linalg.norm(K.toarray(), 2)


def test_time_limit_ends_the_run_and_it_resumes():
    from paper_2508_08062_gb300 import AAPDHGError, Solver, binding
    P = lpgen.tiny()
    tau = _tiny_steps(P)
    with Solver(P, precision="fp64") as s:
        with pytest.raises(AAPDHGError) as e:
            s.set_time_limit(-1.0)
        assert e.value.status == binding.ERR_INVALID
    with Solver(P, precision="fp64") as s:
        s.set_steps(tau, tau)
        s.set_method("aa", mem=5)
        s.set_time_limit(0.005)
        with pytest.raises(AAPDHGError) as e:
            s.iterate(10 ** 7)                     # far more than 5 ms of work
        assert e.value.status == binding.ERR_TIMEOUT
        done = e.value.iters_done
        assert 0 < done < 10 ** 7 and done % 64 == 0
        assert s.counters()["iters"] == done        # not sticky: the handle works
        s.set_time_limit(0.0)
        conv, more = s.iterate(200000, tol=1e-6, kkt_every=64)
        assert conv
        x, y = s.get_iterate()
    # the resumed run is the uninterrupted run: same iterate, bit for bit
    with Solver(P, precision="fp64") as s:
        s.set_steps(tau, tau)
        s.set_method("aa", mem=5)
        conv2, its = s.iterate(200000, tol=1e-6, kkt_every=64)
        x2, y2 = s.get_iterate()
    assert conv2 and its == done + more
    assert np.array_equal(x, x2) and np.array_equal(y, y2)
