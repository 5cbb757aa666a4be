"""Row-block split of one LP over several GPUs: the partition and the
communication schedule of the PDHG step (eq. pdhg) with the Anderson step of
Alg. 2, host side.

Every run of this build has one GPU, so no multi-GPU kernel path exists: the
per-rank work (the half-steps on a block of rows, the memory pass and the mix
on a shard of the iterate) is supplied by a backend object, and this module
plans the split and issues the collectives around it.  The tests drive it on
CPU ranks (gloo) with a stand-in backend and compare the trajectory with the
FP64 oracle.

Partition (K = [G; A] with m rows and n columns; u = (x, y)):
  rank r owns the variables j in [col_lo, col_hi) (rows of K') and the
  constraints i in [row_lo, row_hi) (rows of K), two contiguous blocks
  balanced by nonzeros.  Its shard of every length-(n + m) vector (iterate,
  residual, D-hat, the columns of the Anderson memory) is those two blocks, so
  the memory pass and the AA mix need no communication.
Per loop iteration k:
  1. x-step on the rank's rows of K', which needs all of y^k   -> xh block
  2. all-gather of the (xh, x) pairs                            (2n values)
  3. y-step on the rank's rows of K, which needs all of (xh, x) -> yh block
  4. memory pass on the shard                                   -> partial sums
  5. one all-reduce of the partial sums (SCALARS + 2 m_A values: the
     residual norm, the KKT terms, ||dg||^2, <dg, g>, ||du||^2, the new Gram
     row <dg_s, dg> and the right-hand side <dg_s, g^k> over the memory)
  6. on every rank, from the same sums: the stop test, the safeguard and the
     m_A x m_A solve, so every rank takes the same branch with the same gamma
  7. AA mix on the shard, or the plain step
  8. all-gather of y^{k+1}                                      (m values)
Blocks of unequal size are padded to the largest for the all-gathers.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

# Slots of the all-reduced vector before the 2 m_A memory entries.
SCALARS = ("g2", "dres2", "lam", "cx", "pres2", "qy", "dg2", "dgg", "du2")


def _balanced_cuts(weights, parts):
    """Contiguous cut points (parts + 1) splitting `weights` into parts of
    nearly equal total weight."""
    cum = np.concatenate([[0.0], np.cumsum(np.asarray(weights, dtype=np.float64))])
    targets = cum[-1] * np.arange(1, parts) / parts
    inner = np.searchsorted(cum, targets, side="left")
    cuts = np.concatenate([[0], inner, [len(weights)]]).astype(np.int64)
    return np.maximum.accumulate(cuts)


@dataclass
class RowBlockPlan:
    """Ownership of rows of K' (variables) and rows of K (constraints) by rank."""
    world: int
    m: int
    n: int
    col_cuts: np.ndarray      # world + 1 cut points over the n variables
    row_cuts: np.ndarray      # world + 1 cut points over the m constraints

    def cols(self, r):
        return int(self.col_cuts[r]), int(self.col_cuts[r + 1])

    def rows(self, r):
        return int(self.row_cuts[r]), int(self.row_cuts[r + 1])

    def max_cols(self):
        return int(np.max(np.diff(self.col_cuts)))

    def max_rows(self):
        return int(np.max(np.diff(self.row_cuts)))


def plan_rowblocks(m, n, row_ptr, col_idx, world, row_cost=1.0) -> RowBlockPlan:
    """Contiguous blocks of the rows of K and of K' with nearly equal
    nonzeros (plus row_cost per row for its epilogue) per rank."""
    if world < 1:
        raise ValueError("world >= 1")
    rp = np.asarray(row_ptr, dtype=np.int64)
    row_w = np.diff(rp) + row_cost
    col_w = np.bincount(np.asarray(col_idx, dtype=np.int64), minlength=n) + row_cost
    return RowBlockPlan(world, int(m), int(n), _balanced_cuts(col_w, world),
                        _balanced_cuts(row_w, world))


def allreduce_layout(mem):
    """Offsets in the all-reduced vector: the SCALARS, then the Gram row
    <dg_s, dg> and the right-hand side <dg_s, g^k> over the mem columns."""
    off = {k: i for i, k in enumerate(SCALARS)}
    off["gram_row"] = len(SCALARS)
    off["rhs"] = len(SCALARS) + mem
    off["len"] = len(SCALARS) + 2 * mem
    return off


class Collectives:
    """The two all-gathers and the all-reduce of one iteration over a
    torch.distributed process group (FP64 host or device tensors)."""

    def __init__(self, plan: RowBlockPlan, rank: int, device="cpu"):
        import torch
        import torch.distributed as dist
        self.plan, self.rank, self.dist, self.torch = plan, rank, dist, torch
        self.device = device

    def _gather(self, block, cuts, width):
        torch = self.torch
        pad = np.zeros(width * (1 if block.ndim == 1 else block.shape[1]))
        flat = np.ascontiguousarray(block, dtype=np.float64).reshape(-1)
        pad[:flat.size] = flat
        t = torch.from_numpy(pad).to(self.device)
        outs = [torch.empty_like(t) for _ in range(self.plan.world)]
        self.dist.all_gather(outs, t)
        k = 1 if block.ndim == 1 else block.shape[1]
        parts = [o.cpu().numpy()[:(cuts[r + 1] - cuts[r]) * k] for r, o in enumerate(outs)]
        full = np.concatenate(parts)
        return full if k == 1 else full.reshape(-1, k)

    def gather_x_pairs(self, xh_blk, x_blk):
        """All of (xh, x) from every rank's block (step 2)."""
        both = self._gather(np.stack([xh_blk, x_blk], axis=1), self.plan.col_cuts,
                            self.plan.max_cols())
        return both[:, 0].copy(), both[:, 1].copy()

    def gather_y(self, y_blk):
        """All of y from every rank's block (step 8)."""
        return self._gather(np.asarray(y_blk), self.plan.row_cuts, self.plan.max_rows())

    def allreduce(self, vec):
        """Sum of the ranks' partial sums (step 5)."""
        t = self.torch.from_numpy(np.ascontiguousarray(vec, dtype=np.float64)).to(self.device)
        self.dist.all_reduce(t)
        return t.cpu().numpy()


def run(backend, comm: Collectives, iters, tol=0.0, kkt_every=0):
    """The distributed loop: u^1 = T u^0 and g^0 first (not an iteration), then
    up to `iters` iterations of steps 1-8 above.  backend supplies the rank's
    work on its blocks:
      y_block()                    -> its block of the current y
      x_step(y_full, kkt)          -> (xh block, x block)
      y_step(xh_full, x_full, kkt)    (keeps its yh block)
      memory(kkt, init)            -> partial sums laid out by allreduce_layout
                                      (init: only ||g^0||^2)
      decide(sums, kkt, tol, init) -> "stop", or the branch every rank takes
                                      (init: records ||g^0||, moves to u^1)
      finish(decision)             -> its block of y^{k+1}
    Returns (iterations done, tolerance met)."""
    y_full = comm.gather_y(backend.y_block())
    xh_blk, x_blk = backend.x_step(y_full, False)
    backend.y_step(*comm.gather_x_pairs(xh_blk, x_blk), False)
    backend.decide(comm.allreduce(backend.memory(False, True)), False, tol, True)
    y_full = comm.gather_y(backend.y_block())
    for it in range(iters):
        kkt = kkt_every > 0 and it % kkt_every == 0
        xh_blk, x_blk = backend.x_step(y_full, kkt)
        backend.y_step(*comm.gather_x_pairs(xh_blk, x_blk), kkt)
        decision = backend.decide(comm.allreduce(backend.memory(kkt, False)), kkt, tol, False)
        if decision == "stop":
            return it, True
        y_full = comm.gather_y(backend.finish(decision))
    return iters, False
