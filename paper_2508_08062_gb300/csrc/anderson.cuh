// Anderson part of AA-PDHG (Alg. 2) and FAA-PDHG (Alg. 3-6).
//
// Memory layout: two rings of NSLOT slot-major vectors of length Npad,
//   DG[s] = dg of column s              (the columns of dG^{k-m_k})
//   W[s]  = du + beta D-hat dg          (the columns of dU + beta D-hat dG)
// so the update u_AA = u - H g = u + beta D-hat g - (dU + beta D-hat dG) gamma
// reads one ring.  The Gram matrix dG'dG is kept by slot; each entry is
// formed once, at the first AA attempt after both of its columns exist (the
// Gram pass below), and <dg_s, g^k> is summed at every attempt.
//
// Per iteration (single LP):
//   k_memory   (every iteration, Alg. 2 "for j = 1..m_k"): g^k = uh - u,
//              dg = g^k - g^{k-1}, du = u^k - u^{k-1}; writes the new column
//              and sums ||dg||^2, <dg, g^k>, ||du||^2; its last block appends
//              the column to the list and, when the safeguard failed, ends
//              the iteration (a PDHG step);
//   k_gram     (safeguard passed): the pending Gram entries and the
//              right-hand side in one pass over the columns, then the solve
//              for gamma (Cholesky of dG'dG + eta I; or Reverse, AngleFilter,
//              LengthFilter, Reverse and the QR solve of Alg. 3 from the Gram);
//   k_mix      (AA step accepted): u^{k+1} = P(u + beta D-hat g - W gamma),
//              and du for the next column.  A PDHG step needs no pass: the
//              roles of the two iterate components swap and du = g^k.
#pragma once
#include "common.cuh"
#include "spmv.cuh"

namespace aap {

// ---------------------------------------------------------------------------
// Dense FP64 routines for k <= 32, one warp, matrices in shared memory
// (row-major, leading dimension NSLOT).
// ---------------------------------------------------------------------------

// FP64 issue is scarce on this part (a warp-wide FP64 instruction occupies the
// pipe for many cycles whatever the active lanes), so the dense routines are
// written to issue few FP64 instructions: right-looking Cholesky with one
// reciprocal per pivot and the trailing update spread over the lanes, and
// column-oriented triangular solves.

// Cholesky A = L L' in place (lower triangle), rd[j] = 1 / L[j][j].  Returns
// false when a pivot is not positive (or not finite).
static __device__ bool warp_cholesky(double *A, double *rd, int k) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < k; ++j) {
        const double d = A[j * NSLOT + j];
        if (!(d > 0.0 && isfinite(d))) return false;      // uniform: every lane reads d
        const double piv = sqrt(d), r = 1.0 / piv;
        __syncwarp();
        if (lane == 0) {
            A[j * NSLOT + j] = piv;
            rd[j] = r;
        }
        for (int i = j + 1 + lane; i < k; i += 32) A[i * NSLOT + j] *= r;
        __syncwarp();
        // trailing update of the lower triangle, row i per lane
        for (int i = j + 1 + lane; i < k; i += 32) {
            const double lij = A[i * NSLOT + j];
            for (int l = j + 1; l <= i; ++l) A[i * NSLOT + l] -= lij * A[l * NSLOT + j];
        }
        __syncwarp();
    }
    return true;
}

// Solve L L' x = b (b overwritten by x), column by column; rd = 1 / diag(L).
static __device__ void warp_chol_solve(const double *L, const double *rd, double *b, int k) {
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < k; ++j) {                       // L y = b
        const double yj = b[j] * rd[j];
        __syncwarp();
        if (lane == 0) b[j] = yj;
        for (int i = j + 1 + lane; i < k; i += 32) b[i] -= L[i * NSLOT + j] * yj;
        __syncwarp();
    }
    for (int j = k - 1; j >= 0; --j) {                  // L' x = y
        const double xj = b[j] * rd[j];
        __syncwarp();
        if (lane == 0) b[j] = xj;
        for (int i = lane; i < j; i += 32) b[i] -= L[j * NSLOT + i] * xj;
        __syncwarp();
    }
}

// Shared workspace of the solve.
struct SolveSmem {
    double A[NSLOT * NSLOT];
    double b[NSLOT];
    double rd[NSLOT];
    double sig[NSLOT];
    double bnd[NSLOT];
    double pw[NSLOT + 1];
    int ord[NSLOT];
    int alive[NSLOT];
    int kept[NSLOT];
    int nk;
    int ok;
};

// FAA selection (Alg. 4-6) from the Gram matrix.  Input: list (oldest first,
// k columns).  Output: sm.kept[0..nk) oldest first.  One warp.
static __device__ void faa_select(const DevState *st, int k, double c_s, double kappa, SolveSmem &sm) {
    const int lane = threadIdx.x & 31;
    // Reverse (Alg. 6): newest first
    for (int t = lane; t < k; t += 32) sm.ord[t] = st->list[k - 1 - t];
    __syncwarp();
    for (int idx = lane; idx < k * k; idx += 32) {
        const int a = idx / k, b = idx % k;
        sm.A[a * NSLOT + b] = st->G[sm.ord[a] * NSLOT + sm.ord[b]];
    }
    __syncwarp();
    // AngleFilter (Alg. 4): one QR of F (newest first).  |r_ii| comes from the
    // Cholesky factor of F'F; a column whose distance to the earlier span is
    // below 1e-7 of its norm is treated as dependent (its row of R is zero).
    // sigma_i = |r_ii| / ||f_i||; columns 2..k with sigma_i < c_s are removed.
    for (int j = 0; j < k; ++j) {
        if (lane == 0) {
            const double gjj = sm.A[j * NSLOT + j];
            double d = gjj;
            for (int p = 0; p < j; ++p) d -= sm.A[p * NSLOT + j] * sm.A[p * NSLOT + j];
            double rjj = d > 0.0 ? sqrt(d) : 0.0;
            const double sig = gjj > 0.0 ? rjj / sqrt(gjj) : 0.0;
            sm.sig[j] = sig;
            if (!(sig >= 1e-7)) rjj = 0.0;
            sm.b[j] = rjj;                         // r_jj (0: dependent)
        }
        __syncwarp();
        const double rjj = sm.b[j];
        // row j of R stored in the upper triangle: R[j][i] for i > j
        for (int i = j + 1 + lane; i < k; i += 32) {
            double s = sm.A[j * NSLOT + i];
            for (int p = 0; p < j; ++p) s -= sm.A[p * NSLOT + j] * sm.A[p * NSLOT + i];
            sm.A[j * NSLOT + i] = rjj > 0.0 ? s / rjj : 0.0;
        }
        if (lane == 0) sm.A[j * NSLOT + j] = rjj;
        __syncwarp();
    }
    // Note: the lower triangle of sm.A still holds F'F entries; the diagonal
    // was overwritten, so ||f_i||^2 is re-read from the Gram below.
    if (lane == 0) {
        int na = 0;
        for (int i = 0; i < k; ++i)
            if (i == 0 || !(sm.sig[i] < c_s)) sm.alive[na++] = i;
        // LengthFilter (Alg. 5) over the surviving columns (newest first):
        // b_j of Proposition 1.2 from ||f_j||, and e_j = ||du_j||.
        const double c_t = sqrt(1.0 - c_s * c_s);
        const double rho2 = ((c_t + c_s) / c_s) * ((c_t + c_s) / c_s);
        sm.pw[0] = 1.0;
        for (int e = 1; e <= na; ++e) sm.pw[e] = sm.pw[e - 1] * rho2;   // ((c_t+c_s)/c_s)^(2e)
        double f2[NSLOT];
        for (int t = 0; t < na; ++t) {
            const int sl = sm.ord[sm.alive[t]];
            f2[t] = st->G[sl * NSLOT + sl];
        }
        for (int j = 1; j <= na; ++j) {
            double bj;
            if (j == 1) {
                bj = 1.0 / f2[0];
            } else {
                // c_t^2 (c_t+c_s)^{2(j-2)} / (||f_1||^2 c_s^{2(j-2)})
                double s = c_t * c_t * sm.pw[j - 2] / f2[0];
                // sum_{i=2}^{j-1} c_t^2 (c_t+c_s)^{2(j-i-1)} / (||f_i||^2 c_s^{2(j-i)})
                for (int i = 2; i <= j - 1; ++i)
                    s += c_t * c_t * sm.pw[j - i - 1] / (f2[i - 1] * c_s * c_s);
                s += 1.0 / f2[j - 1];
                bj = s / (c_s * c_s);
            }
            sm.bnd[j - 1] = bj;
        }
        int mbar = 0;
        for (int kk = na; kk >= 1; --kk) {
            double se = 0.0, sb = 0.0;
            for (int j = 0; j < kk; ++j) {
                se += st->en2[sm.ord[sm.alive[j]]];
                sb += sm.bnd[j];
            }
            if (se * sb <= kappa * kappa) { mbar = kk; break; }
        }
        // keep the first mbar (newest) survivors; Reverse back to oldest first
        for (int t = 0; t < mbar; ++t) sm.kept[t] = sm.ord[sm.alive[mbar - 1 - t]];
        sm.nk = mbar;
    }
    __syncwarp();
}

// Solve for gamma over columns cols[0..k) (oldest first): Cholesky of the
// Gram block + eta I.  Writes st->use / st->gamma.  One warp.  Returns ok.
static __device__ bool gram_solve(DevState *st, const int *cols, int k, double eta, SolveSmem &sm) {
    const int lane = threadIdx.x & 31;
    for (int idx = lane; idx < k * k; idx += 32) {
        const int a = idx / k, b = idx % k;
        sm.A[a * NSLOT + b] = st->G[cols[a] * NSLOT + cols[b]] + (a == b ? eta : 0.0);
    }
    for (int t = lane; t < k; t += 32) sm.b[t] = st->rhs[cols[t]];
    __syncwarp();
    const bool ok = warp_cholesky(sm.A, sm.rd, k);
    __syncwarp();
    if (ok) {
        warp_chol_solve(sm.A, sm.rd, sm.b, k);
        __syncwarp();
        bool fin = true;
        for (int t = 0; t < k; ++t) fin = fin && isfinite(sm.b[t]);
        if (!fin) return false;
        for (int t = lane; t < k; t += 32) {
            st->use[t] = cols[t];
            st->gamma[t] = sm.b[t];
        }
        if (lane == 0) st->use_count = k;
    }
    return ok;
}

// The rest of an iteration's m x m work once the Gram matrix, the right-hand
// side and the column list are current, run by warp 0 of one block: when the
// safeguard passed (st->want_aa), the solve of Alg. 2 or the filters and
// solve of Alg. 3; then the slot for the next column, the counters and the
// trace.
static __device__ void memory_solve_tail(DevState *st, const MethodParams &mp, int M, SolveSmem &sm,
                                  const Trace &tr) {
    const int lane = threadIdx.x & 31;
    int accept = 0, lsfail = 0;
    if (M > 0) {
        if (st->want_aa) {
            const int k = st->count;
            if (mp.method == 1) {
                sm.nk = k;
                for (int t = lane; t < k; t += 32) sm.kept[t] = st->list[t];
                __syncwarp();
                const bool ok = gram_solve(st, sm.kept, k, mp.eta, sm);
                accept = ok ? 1 : 0;
                lsfail = ok ? 0 : 1;
            } else {
                faa_select(st, k, mp.c_s, mp.kappa, sm);
                const int nk = sm.nk;
                bool ok = true;
                if (nk > 0) ok = gram_solve(st, sm.kept, nk, 0.0, sm);
                else if (lane == 0) st->use_count = 0;
                __syncwarp();
                accept = ok ? 1 : 0;
                lsfail = ok ? 0 : 1;
                if (ok && mp.faa_adaptive) {
                    for (int t = lane; t < nk; t += 32) st->list[t] = sm.kept[t];
                    if (lane == 0) st->count = nk;
                }
            }
        }
        __syncwarp();
        // slot for the next column's du: the lowest slot not in the list
        const int cnt = st->count;
        unsigned long long used = 0ull;
        for (int t = lane; t < cnt; t += 32) used |= 1ull << st->list[t];
#pragma unroll
        for (int o = 16; o; o >>= 1) used |= __shfl_xor_sync(0xffffffffu, used, o);
        if (lane == 0) st->free_slot = __ffsll((long long)~used) - 1;
    }
    if (lane == 0) {
        const int64_t it = st->it;
        st->accept = accept;
        if (accept) st->n_aa += 1; else st->n_pd += 1;
        if (lsfail) st->n_lsfail += 1;
        if (it < tr.cap) {
            tr.branch[it] = (int8_t)(accept ? 1 : (lsfail ? 2 : 0));
            tr.mk[it] = accept ? st->use_count : -1;
        }
        st->it = it + 1;
    }
}

// The ring's columns are read in groups of COLGRP with all loads of a group
// issued before their use.
constexpr int COLGRP = 8;

// ---------------------------------------------------------------------------
// Single-LP memory pass, in two kernels.
//
// k_memory (every iteration) forms g^k = uh - u, dg = g^k - g^{k-1} and
// du = u^k - u^{k-1}, writes the new memory column (dg, and du + beta D-hat
// dg), and sums ||dg||^2, <dg, g^k> and ||du||^2.  Its last block appends the
// column to the list (dropping the oldest when m_A are held).  The new
// column's Gram entries with the older columns are formed later, by k_gram,
// at the first AA attempt that needs them (the safeguard of Alg. 2 passing):
// until then the column is "stale", and a column that leaves the memory while
// stale never has them formed.  When the safeguard failed, the iteration ends
// in k_memory's last block (a PDHG step).
//
// k_gram (only when the safeguard passed) forms, in one pass over the memory
// columns and g^k, the entries <dg_s, dg_t> of every stale column s with every
// other column t and the right-hand side <dg_t, g^k> of every column, then
// solves (Alg. 2, or the filters of Alg. 3) in its last block.  Every Gram
// entry is one dot product of two stored columns, formed once, as in the
// Gram update of Sec. 5 (one new row per column): with an attempt at every
// iteration k_gram forms one row per iteration; with r failed safeguard
// tests in between it forms the r rows in one pass instead of r passes, and
// none in iterations without an attempt.
// ---------------------------------------------------------------------------

// Per-element work of k_memory on W consecutive elements at e0:
// acc[0] ||dg||^2, acc[1] <dg, g^k>, acc[2] ||du||^2; GN: acc[3] ||g^k||^2
// (the batched path forms the safeguard's residual norm here).
template <typename V, int W, bool GN = false>
__device__ __forceinline__ void push_elems(const Prob<V> &P, int64_t e0, int cur, bool prev_acc,
                                           V beta, V *DGn, V *Wn, Acc<V> (&acc)[GN ? 4 : 3]) {
    const V *UPs = reinterpret_cast<const V *>(P.UP);
    const Pack<V, W> pa = ld_stream<V, W>(UPs + 2 * e0), pb = ld_stream<V, W>(UPs + 2 * e0 + W);
    const Pack<V, W> gp = ld_stream<V, W>(P.g + e0);
    const Pack<V, W> dh = ld<V, W>(P.dh + e0);
    Pack<V, W> wn;
    if (prev_acc) wn = ld_stream<V, W>(Wn + e0);
    Pack<V, W> gk, dgk, wk;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const int i0 = 2 * i, i1 = 2 * i + 1;
        const V c0 = i0 < W ? pa.v[i0 % W] : pb.v[i0 % W];
        const V c1 = i1 < W ? pa.v[i1 % W] : pb.v[i1 % W];
        const V u = cur ? c1 : c0, uh = cur ? c0 : c1;
        const V g = uh - u;
        const V dg = g - gp.v[i];
        const V du = prev_acc ? wn.v[i] : gp.v[i];     // u^k - u^{k-1}
        gk.v[i] = g;
        dgk.v[i] = dg;
        wk.v[i] = du + beta * dh.v[i] * dg;
        acc[0].add_sq(dg);
        acc[1].add_prod(dg, g);
        acc[2].add_sq(du);
        if constexpr (GN) acc[3].add_sq(g);
    }
    st<V, W>(P.g + e0, gk);
    st<V, W>(DGn + e0, dgk);
    st<V, W>(Wn + e0, wk);
}

// Appends the new column (warp 0 of k_memory's last block) and, when the
// safeguard failed, ends the iteration.  red = {||dg||^2, <dg, g^k>, ||du||^2}.
static __device__ void push_finalize(DevState *st, const MethodParams &mp, int M, int sn, const double *red,
                              SolveSmem &sm, const Trace &tr) {
    const int lane = threadIdx.x & 31;
    if (M > 0 && lane == 0) {
        int cnt = st->count;
        if (cnt == M) {                                 // the oldest column leaves
            st->stale &= ~(1ull << st->list[0]);
            for (int i = 1; i < cnt; ++i) st->list[i - 1] = st->list[i];
            cnt -= 1;
        }
        st->list[cnt] = sn;
        st->count = cnt + 1;
        st->new_slot = sn;
        st->G[sn * NSLOT + sn] = red[0];
        st->rhs[sn] = red[1];
        st->en2[sn] = red[2];
        if (cnt > 0) st->stale |= 1ull << sn;           // entries with the older columns pending
    }
    __syncwarp();
    if (M > 0 && st->want_aa) return;                   // k_gram finishes the iteration
    memory_solve_tail(st, mp, M, sm, tr);
}

// k_memory: see above.  mode INIT: only g^0 = u^1 - u^0 is written.
// fin = 1 (iterations without a KKT test): the half-steps' final reduction
// (||g^k||, the safeguard test; k_finalize's work) runs here too.  Without a
// KKT test the iteration cannot stop, and the streaming part neither reads
// nor writes what that reduction does, so the two run side by side: the grid
// has one block more than P.grid3, and that block runs the reduction while
// blocks 0 .. P.grid3 - 1 stream (on the restart path, which has no streaming
// sums, it streams too and the last block runs the reduction).  A NaN/Inf the
// reduction finds still stops the run before any AA step.
template <typename V>
__global__ void __launch_bounds__(BLOCK) k_memory(Prob<V> P, MethodParams mp, int mode, int fin) {
    constexpr int W = 16 / sizeof(V);
    DevState *st = P.st;
    if (st->done | st->error) return;
    const int M = (mp.method == 0) ? 0 : mp.mem;
    __shared__ int s_new, s_prev_acc;
    __shared__ typename Acc<V>::Packed sh[WARPS * 3];
    __shared__ double red[3];
    __shared__ SolveSmem sm;
    const int cur = (mode == MODE_INIT) ? 0 : (int)(st->it & 1) ^ 1;
    // the iteration of a primal weight update restarts the memory: a plain
    // step, g^k kept as the previous residual, no column formed across it
    const bool restart = mode == MODE_ITER && st->restart;

    if (mode == MODE_INIT || restart) {
        if (M > 0) {
            for (int64_t e = blockIdx.x * (int64_t)BLOCK + threadIdx.x; e < P.N;
                 e += (int64_t)gridDim.x * BLOCK) {
                const typename Vec2<V>::T pr = P.UP[e];
                P.g[e] = comp<V>(pr, 1 - cur) - comp<V>(pr, cur);
            }
        }
        if (!last_block(&st->cnt_ring)) return;
        if (fin) {
            finalize_T<V>(P, mp, MODE_ITER, false);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            st->count = 0;
            st->stale = 0ull;
            st->want_aa = 0;  // a restart takes the plain step
            st->new_slot = 0;
            st->free_slot = 0;
            st->accept = 0;   // u^1 = T u^0 behaves as a PDHG step: du^0 = g^0
            st->use_count = 0;
            if (restart) {
                const int64_t it = st->it;
                st->n_pd += 1;
                st->restart = 0;
                if (it < P.tr.cap) {
                    P.tr.branch[it] = 0;
                    P.tr.mk[it] = -1;
                }
                st->it = it + 1;
            } else {
                st->it = 0;
                st->init_done = 1;
            }
        }
        return;
    }

    if (threadIdx.x == 0) {
        s_new = st->free_slot;
        s_prev_acc = st->accept;
    }
    __syncthreads();
    const int sn = s_new;
    const bool prev_acc = s_prev_acc != 0;
    const bool fin_block = blockIdx.x >= P.grid3;        // the extra block (fin = 1 only)
    if (fin_block) {
        finalize_T<V>(P, mp, mode, false);
    } else if (M > 0) {
        Acc<V> acc[3];
        V *DGn = P.DG + (int64_t)sn * P.Npad;
        V *Wn = P.W + (int64_t)sn * P.Npad;
        const V beta = (V)mp.beta;
        const int64_t NV = P.N / W * W;
        const int64_t stride = (int64_t)P.grid3 * BLOCK;
        for (int64_t e0 = (blockIdx.x * (int64_t)BLOCK + threadIdx.x) * W; e0 < NV; e0 += stride * W)
            push_elems<V, W>(P, e0, cur, prev_acc, beta, DGn, Wn, acc);
        for (int64_t e = NV + blockIdx.x * (int64_t)BLOCK + threadIdx.x; e < P.N; e += stride)
            push_elems<V, 1>(P, e, cur, prev_acc, beta, DGn, Wn, acc);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            acc[j].warp_allreduce();
            if (lane == 0) sh[warp * 3 + j] = acc[j].pack();
        }
        __syncthreads();
        if (threadIdx.x < 3) {
            double v = 0.0;
            for (int w = 0; w < WARPS; ++w) v += Acc<V>::unpack(sh[w * 3 + threadIdx.x]);
            P.part3[(int64_t)blockIdx.x * 3 + threadIdx.x] = v;
        }
    }
    if (!last_block(&st->cnt_ring)) return;
    if (fin) {
        if ((int)gridDim.x == P.grid3) {                 // no extra block (M = 0)
            finalize_T<V>(P, mp, mode, false);
            __syncthreads();
        }
        if (*reinterpret_cast<volatile int32_t *>(&st->error)) return;
    }
    if (M > 0) {
        // one warp per partial column, lanes striding the blocks: fixed order
        const int wl = threadIdx.x & 31, ww = threadIdx.x >> 5;
        if (ww < 3) {
            double v = 0.0;
            for (int b = wl; b < P.grid3; b += 32) v += __ldcg(P.part3 + (int64_t)b * 3 + ww);
#pragma unroll
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (wl == 0) red[ww] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    push_finalize(st, mp, M, sn, red, sm, P.tr);
}

// k_gram: see above.  The pairs of vectors to multiply (columns by list
// position 0 .. k-1, and k for g^k) are listed in shared memory.  The block is
// warp-specialised: warp 0 brings tiles of GRAM_TILE_BYTES of every vector
// into shared memory with bulk asynchronous copies (cp.async.bulk), each stage
// completing on its "full" mbarrier, up to GRAM_STAGES tiles ahead; the other
// GRAM_CWARPS warps multiply, consumer warp c accumulating pairs c, c +
// GRAM_CWARPS, ... (at most GRAM_PW per warp and pass; more pairs take more
// passes over the tiles) in float-float pairs (mixed) or FP64, and release a
// stage by arriving on its "empty" mbarrier.  The elements after the last
// whole tile are read directly by block 0.  Block partials go to
// part4[block][pair]; the last block sums them in block order, writes the
// Gram entries and the right-hand side, and solves.  Every wait on a barrier
// is bounded: one that gives up sets st->error = 2 (reported by the host),
// and the block waits (bounded) for its copies in flight before it returns.
constexpr int GRAM_PW = 16;
constexpr int GRAM_MAX_OCC = 8;            // resident blocks per SM the Gram pass uses at most
constexpr int GRAM_MAXPAIRS = MAXM * (MAXM - 1) / 2 + MAXM;
constexpr int GRAM_TILE_BYTES = 2048;
constexpr int GRAM_STAGES = 2;
constexpr int GRAM_CWARPS = WARPS - 1;     // consumer warps (warp 0 produces)
constexpr int GRAM_WAIT_LIMIT = 1 << 22;   // try_wait polls before a wait gives up

__host__ __device__ constexpr int gram_dyn_smem(int mem) {
    return GRAM_STAGES * (mem + 1) * GRAM_TILE_BYTES;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
}

// Bounded wait for the phase with parity `parity` of the barrier to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    for (int it = 0; it < GRAM_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(d), "l"(src), "r"(bytes), "r"(b)
        : "memory");
}

// The Gram pass's work list for one LP with k columns list[0..k) (oldest
// first), `stale` the slots whose entries with the other columns are pending:
// every pair (a, b), a < b < k, of list positions with a stale column, then
// the pairs (a, k), a < k - 1, of a column with g^k (position k).  The
// right-hand side <dg_s, g^k> is always summed directly: carried as
// <dg_s, g^{k-1}> + <dg_s, dg> (the update of Sec. 5) it loses its relative
// accuracy to cancellation once g^k is much smaller than g^{k-1}.  The newest
// column's <dg, g^k> comes from the memory pass.  Returns the pair count.
// One thread.
static __device__ int gram_pair_list(const int *list, int k, uint64_t stale, int16_t *pa, int16_t *pb) {
    int np = 0;
    for (int a = 0; a < k; ++a)
        for (int b = a + 1; b < k; ++b)
            if (((stale >> list[a]) | (stale >> list[b])) & 1ull) {
                pa[np] = (int16_t)a;
                pb[np] = (int16_t)b;
                ++np;
            }
    for (int a = 0; a + 1 < k; ++a) {
        pa[np] = (int16_t)a;
        pb[np] = (int16_t)k;
        ++np;
    }
    return np;
}

// Gram entries and right-hand side from the pair values v[0..np) of
// gram_pair_list, then the stale set cleared.  One warp (lanes stride the
// pairs).
static __device__ void gram_store(DevState *st, const int *list, int k, const int16_t *pa,
                                  const int16_t *pb, int np, const double *v) {
    const int lane = threadIdx.x & 31;
    for (int p = lane; p < np; p += 32) {
        const int a = list[pa[p]], bv = pb[p];
        if (bv == k) {
            st->rhs[a] = v[p];
        } else {
            const int b = list[bv];
            st->G[a * NSLOT + b] = v[p];
            st->G[b * NSLOT + a] = v[p];
        }
    }
    __syncwarp();
    if (lane == 0) st->stale = 0ull;
    __syncwarp();
}

template <typename V>
__global__ void __launch_bounds__(BLOCK) k_gram(Prob<V> P, MethodParams mp) {
    constexpr int W = 16 / sizeof(V);
    constexpr int TILE = GRAM_TILE_BYTES / sizeof(V);   // elements per tile
    constexpr int VPL = TILE / (32 * W);                // 16-byte vectors per lane and tile
    DevState *st = P.st;
    if (st->done | st->error) return;
    if (!st->want_aa || mp.method == 0 || mp.mem == 0) return;
    extern __shared__ __align__(128) unsigned char gram_smem[];
    __shared__ int s_k, s_np, s_fail;
    __shared__ int s_list[NSLOT];
    __shared__ uint64_t s_stale;
    __shared__ int16_t s_pa[GRAM_MAXPAIRS], s_pb[GRAM_MAXPAIRS];
    __shared__ const V *s_vec[NSLOT + 1];
    __shared__ __align__(8) uint64_t full[GRAM_STAGES], empty[GRAM_STAGES];
    __shared__ SolveSmem sm;
    if (threadIdx.x == 0) {
        s_k = st->count;
        s_stale = st->stale;
        s_fail = 0;
    }
    if (threadIdx.x < NSLOT) s_list[threadIdx.x] = st->list[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {                              // the pair list, from shared memory
        s_np = gram_pair_list(s_list, s_k, s_stale, s_pa, s_pb);
        for (int s2 = 0; s2 < GRAM_STAGES; ++s2) {
            mbar_init(&full[s2], 1);
            mbar_init(&empty[s2], GRAM_CWARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int k = s_k, np = s_np;
    if (threadIdx.x < k) s_vec[threadIdx.x] = P.DG + (int64_t)s_list[threadIdx.x] * P.Npad;
    if (threadIdx.x == k) s_vec[k] = P.g;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nfull = P.N / TILE;                   // whole tiles, copied in bulk
    const int64_t mine = nfull > blockIdx.x ? (nfull - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int npass = (np + GRAM_CWARPS * GRAM_PW - 1) / (GRAM_CWARPS * GRAM_PW);
    const int64_t items = mine * npass;                 // (pass, tile), in order
    auto stage_ptr = [&](int s2, int v) {
        return reinterpret_cast<V *>(gram_smem + ((size_t)s2 * (k + 1) + v) * GRAM_TILE_BYTES);
    };

    if (warp == 0) {
        // producer: item q into stage q % GRAM_STAGES once its consumers released it
        if (lane == 0) {
            for (int64_t q = 0; q < items; ++q) {
                const int s2 = (int)(q % GRAM_STAGES);
                if (q >= GRAM_STAGES && !mbar_wait(&empty[s2], (uint32_t)(((q / GRAM_STAGES) - 1) & 1))) {
                    s_fail = 1;
                    break;
                }
                const int64_t e0 = (blockIdx.x + (q % mine) * gridDim.x) * (int64_t)TILE;
                mbar_expect_tx(&full[s2], (uint32_t)((k + 1) * GRAM_TILE_BYTES));
                for (int v = 0; v <= k; ++v)
                    bulk_g2s(stage_ptr(s2, v), s_vec[v] + e0, GRAM_TILE_BYTES, &full[s2]);
            }
            // every copy issued must land before the block may leave
            const int64_t last = items < GRAM_STAGES ? items : GRAM_STAGES;
            for (int64_t j = 0; j < last; ++j) {
                const int64_t q = items - 1 - j;
                if (!mbar_wait(&full[q % GRAM_STAGES], (uint32_t)((q / GRAM_STAGES) & 1))) s_fail = 1;
            }
        }
    } else {
        const int cw = warp - 1;
        for (int pass = 0; pass < npass; ++pass) {
            const int p0 = pass * GRAM_CWARPS * GRAM_PW;
            Acc<V> acc[GRAM_PW];
            for (int64_t i = 0; i < mine; ++i) {
                const int64_t q = (int64_t)pass * mine + i;
                const int s2 = (int)(q % GRAM_STAGES);
                if (!mbar_wait(&full[s2], (uint32_t)((q / GRAM_STAGES) & 1))) {
                    if (lane == 0) s_fail = 1;
                    break;
                }
#pragma unroll
                for (int j = 0; j < GRAM_PW; ++j) {
                    const int p = p0 + cw + j * GRAM_CWARPS;
                    if (p < np) {
                        const V *a = stage_ptr(s2, s_pa[p]), *b = stage_ptr(s2, s_pb[p]);
#pragma unroll
                        for (int c = 0; c < VPL; ++c) {
                            const int off = (c * 32 + lane) * W;
                            const Pack<V, W> x = ld<V, W>(a + off), y = ld<V, W>(b + off);
#pragma unroll
                            for (int t = 0; t < W; ++t) acc[j].add_prod(x.v[t], y.v[t]);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s2]);
            }
            // the elements after the last whole tile, read directly by block 0
            if (blockIdx.x == 0) {
#pragma unroll
                for (int j = 0; j < GRAM_PW; ++j) {
                    const int p = p0 + cw + j * GRAM_CWARPS;
                    if (p < np) {
                        const V *a = s_vec[s_pa[p]], *b = s_vec[s_pb[p]];
                        for (int64_t e = nfull * TILE + lane; e < P.N; e += 32) acc[j].add_prod(a[e], b[e]);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < GRAM_PW; ++j) {
                const int p = p0 + cw + j * GRAM_CWARPS;
                if (p < np) {
                    acc[j].warp_allreduce();
                    if (lane == 0) P.part4[(int64_t)blockIdx.x * GRAM_MAXPAIRS + p] = acc[j].value();
                }
            }
        }
    }
    __syncthreads();
    if (s_fail) {
        if (threadIdx.x == 0) st->error = 2;
        return;
    }
    if (!last_block(&st->cnt_gram)) return;
    // one warp per pair, lanes striding the blocks: fixed order
    for (int p = warp; p < np; p += WARPS) {
        double v = 0.0;
        for (int b = lane; b < P.grid4; b += 32) v += __ldcg(P.part4 + (int64_t)b * GRAM_MAXPAIRS + p);
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) {
            const int a = s_list[s_pa[p]], bv = s_pb[p];
            if (bv == k) {
                st->rhs[a] = v;
            } else {
                const int b = s_list[bv];
                st->G[a * NSLOT + b] = v;
                st->G[b * NSLOT + a] = v;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x >= 32) return;
    if (lane == 0) st->stale = 0ull;
    __syncwarp();
    memory_solve_tail(st, mp, mp.mem, sm, P.tr);
}

// ---------------------------------------------------------------------------
// k_mix: u^{k+1} = P(u^k + beta D-hat g^k - sum_t gamma_t W[use_t]) written
// over T(u^k), and du = u^{k+1} - u^k into the free slot (Alg. 2, the AA
// branch; the projection P of Sec. 3 is a clamp to [lo, hi]).
// ---------------------------------------------------------------------------
template <typename V, int MC, int W>
__device__ __forceinline__ void mix_elems(const Prob<V> &P, int64_t e0, int cur, V beta,
                                          const V *gam, const int64_t *off, int k, V *Wf) {
    V *UPs = reinterpret_cast<V *>(P.UP);
    Pack<V, W> pa = ld<V, W>(UPs + 2 * e0), pb = ld<V, W>(UPs + 2 * e0 + W);
    const Pack<V, W> dh = ld<V, W>(P.dh + e0);
    const Pack<V, W> lo = ld<V, W>(P.lo + e0), hi = ld<V, W>(P.hi + e0);
    V u[W], v[W];
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const int i0 = 2 * i, i1 = 2 * i + 1;
        const V c0 = i0 < W ? pa.v[i0 % W] : pb.v[i0 % W];
        const V c1 = i1 < W ? pa.v[i1 % W] : pb.v[i1 % W];
        u[i] = cur ? c1 : c0;
        const V uh = cur ? c0 : c1;
        v[i] = u[i] + beta * dh.v[i] * (uh - u[i]);
    }
#pragma unroll
    for (int t0 = 0; t0 < MC; t0 += COLGRP) {
        if (t0 >= k) break;
        Pack<V, W> col[COLGRP];
#pragma unroll
        for (int j = 0; j < COLGRP; ++j)
            if (t0 + j < MC && t0 + j < k) col[j] = ld_stream<V, W>(P.W + off[t0 + j] + e0);
#pragma unroll
        for (int j = 0; j < COLGRP; ++j)
            if (t0 + j < MC && t0 + j < k)
#pragma unroll
                for (int i = 0; i < W; ++i) v[i] = fma(-gam[t0 + j], col[j].v[i], v[i]);
    }
    Pack<V, W> du;
#pragma unroll
    for (int i = 0; i < W; ++i) {
        V x = v[i] < lo.v[i] ? lo.v[i] : (v[i] > hi.v[i] ? hi.v[i] : v[i]);
        du.v[i] = x - u[i];
        const int slot = 2 * i + (1 - cur);             // overwrite T(u^k) with u^{k+1}
        if (slot < W) pa.v[slot % W] = x; else pb.v[slot % W] = x;
    }
    st<V, W>(UPs + 2 * e0, pa);
    st<V, W>(UPs + 2 * e0 + W, pb);
    st<V, W>(Wf + e0, du);
}

template <typename V, int MC>
__global__ void __launch_bounds__(BLOCK) k_mix(Prob<V> P, MethodParams mp) {
    constexpr int W = 16 / sizeof(V);
    DevState *st = P.st;
    if (st->done | st->error) return;
    if (!st->accept) return;
    __shared__ V s_gam[MC];
    __shared__ int64_t s_off[MC];
    __shared__ int s_k, s_free;
    if (threadIdx.x == 0) {
        s_k = st->use_count;
        s_free = st->free_slot;
    }
    if (threadIdx.x < MC) {
        const bool on = threadIdx.x < st->use_count;
        s_gam[threadIdx.x] = on ? (V)st->gamma[threadIdx.x] : V(0);
        s_off[threadIdx.x] = (int64_t)(on ? st->use[threadIdx.x] : 0) * P.Npad;
    }
    __syncthreads();
    const int k = s_k;
    // the iteration counter was already advanced by k_memory
    const int cur = (int)(st->it & 1);
    const V beta = (V)mp.beta;
    V *Wf = P.W + (int64_t)s_free * P.Npad;
    const int64_t NV = P.N / W * W;
    const int64_t stride = (int64_t)gridDim.x * BLOCK;
    for (int64_t e0 = (blockIdx.x * (int64_t)BLOCK + threadIdx.x) * W; e0 < NV; e0 += stride * W)
        mix_elems<V, MC, W>(P, e0, cur, beta, s_gam, s_off, k, Wf);
    for (int64_t e = NV + blockIdx.x * (int64_t)BLOCK + threadIdx.x; e < P.N; e += stride)
        mix_elems<V, MC, 1>(P, e, cur, beta, s_gam, s_off, k, Wf);
}

}  // namespace aap
