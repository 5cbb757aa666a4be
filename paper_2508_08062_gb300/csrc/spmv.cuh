// Fused PDHG half-steps (Sec. 3, eq. pdhg) on row-sliced CSR matrices.
//
// Both K and K' are stored with rows renumbered longest first.  Rows longer
// than SELL_MAX entries are read as CSR in chunks of LONG_CHUNK entries, one
// warp per chunk with coalesced loads; the warp that finishes the last chunk
// of a row sums the chunk partials in chunk order (deterministic) and runs the
// row epilogue.  Shorter rows are stored as SELL-32 slices (32 rows of
// similar length, column by column): a warp reads one slice with fully
// coalesced, mutually independent index/value loads and issues all gathers of
// a step together, lane = row, so the epilogue is coalesced too.
//
// The x-step kernel computes, per variable j,
//     s_j = (K'y)_j,  xh_j = P_X(x_j - tau (c_j - s_j))
// and the y-step kernel, per constraint i,
//     z_i = (K(2 xh - x))_i,  yh_i = P_Y(y_i + sigma (q_i - z_i)),
// with the reflection 2 xh - x formed from the (xh, x) pair gathered once.
// Their epilogues accumulate ||g^k||^2 (g = T u - u) and, on KKT iterations,
// the terms of the relative KKT residual (Remark on termination conditions)
// at the current iterate u^k: ||c - K'y - lambda||^2 with lambda = P_Lambda(
// c - K'y), l'lambda+ - u'lambda-, c'x (x-step) and the primal violation
// ||(q - Kx)_{=}, (q - Kx)_{>=,+}||^2 and q'y (y-step, which then also
// accumulates K x^k in the same pass).
#pragma once
#include "common.cuh"

namespace aap {

// Process warp task t of matrix A.  gather(col, val, acc) folds one entry
// into the NACC per-lane partial sums.  The epilogue has three parts:
// epi.skip(problem) says that a problem's rows are left untouched (a batch
// member that has stopped), epi.pre(row, problem) loads the row's own inputs
// (issued before the sum, since they do not depend on it) and
// epi(row, pre, sums) finishes the row on one lane.  Epi::kRowOrder: the
// slices are those of one LP in row order (slice q holds rows n_long + 32q
// on), so a lane's row is known without the slice's metadata and its inputs
// are requested together with that metadata; otherwise (a batch) the row
// comes from the metadata.
template <typename V, int NACC, int G = SLICES_PER_TASK, int LD = LOADS, class Gather, class Epi>
__device__ __forceinline__ void run_task(const CSRView<V> &A, int64_t t, Gather &gather, Epi &epi) {
    typedef typename Epi::Pre Pre;
    const int lane = threadIdx.x & 31;

    if (t < A.n_chunks) {                               // chunk of a long row
        V acc[NACC];
#pragma unroll
        for (int a = 0; a < NACC; ++a) acc[a] = V(0);
        const int chunk = (int)t;
        int4 cm;
        if constexpr (Epi::kRowOrder) {          // one LP: long-row id = row, problem 0
            cm.x = __ldg(reinterpret_cast<const int *>(A.chunk_meta + chunk));
            cm.y = cm.x;
            cm.z = 0;
        } else {
            cm = __ldg(A.chunk_meta + chunk);
        }
        const int r = cm.x, lr = cm.y;
        if (epi.skip(cm.z)) return;
        const int c0 = __ldg(A.row_chunk0 + lr);
        const int nch = __ldg(A.row_chunk0 + lr + 1) - c0;
        const int k0 = __ldg(A.rp + r) + (chunk - c0) * A.long_chunk;
        const int k1 = min(k0 + A.long_chunk, __ldg(A.rp + r + 1));
        Pre pre;
        if (nch == 1 && lane == 0) pre = epi.pre(r, cm.z);
        for (int kb = k0 + lane; kb < k1; kb += 32 * LD) {
            int ci[LD];
            V va[LD];
#pragma unroll
            for (int j = 0; j < LD; ++j) {
                const int k = kb + 32 * j;
                ci[j] = k < k1 ? __ldcs(A.ci + k) : 0;
                va[j] = k < k1 ? __ldcs(A.val + k) : V(0);
            }
#pragma unroll
            for (int j = 0; j < LD; ++j)
                if (kb + 32 * j < k1) gather(ci[j], va[j], acc);
        }
#pragma unroll
        for (int a = 0; a < NACC; ++a)
#pragma unroll
            for (int o = 16; o; o >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
        if (nch == 1) {
            if (lane == 0) epi(r, pre, acc);
            return;
        }
        int last = 0;
        if (lane == 0) {
#pragma unroll
            for (int a = 0; a < NACC; ++a) A.chunk_part[(int64_t)chunk * 2 + a] = acc[a];
            __threadfence();
            last = (atomicAdd(A.chunk_cnt + lr, 1u) == (unsigned)(nch - 1));
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last && lane == 0) {
            __threadfence();
            pre = epi.pre(r, cm.z);
            V tot[NACC];
#pragma unroll
            for (int a = 0; a < NACC; ++a) tot[a] = V(0);
            for (int c = c0; c < c0 + nch; ++c)
#pragma unroll
                for (int a = 0; a < NACC; ++a) tot[a] += __ldcg(A.chunk_part + (int64_t)c * 2 + a);
            A.chunk_cnt[lr] = 0u;
            epi(r, pre, tot);
        }
        return;
    }

    // G SELL-32 slices in lockstep: lane = row of each slice, entry tt of a
    // slice's 32 rows contiguous; padding entries are zeros.
    constexpr int B = LD / G;
    const int sl0 = (int)(t - A.n_chunks) * G;
    int2 meta[G];
    int r[G];
    bool valid[G];
    Pre pre[G];
    V acc[G][NACC];
    int wmax = 0;
    if constexpr (Epi::kRowOrder) {
        // one LP: rows from the slice index, only (offset, width) loaded
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const bool on = sl0 + g < A.n_slices;
            meta[g] = on ? __ldg(reinterpret_cast<const int2 *>(A.slice_meta + sl0 + g)) : make_int2(0, 0);
            r[g] = A.n_long + (sl0 + g) * 32 + lane;
            if (r[g] < A.rows) pre[g] = epi.pre(r[g], 0);
#pragma unroll
            for (int a = 0; a < NACC; ++a) acc[g][a] = V(0);
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            meta[g].x += lane;
            wmax = max(wmax, meta[g].y);
            valid[g] = r[g] < A.rows;
        }
    } else {
        // a batch: rows and problem from the slice's metadata
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const bool on = sl0 + g < A.n_slices;
            const int4 m4 = on ? __ldg(A.slice_meta + sl0 + g) : make_int4(0, 0, 0, 0);
            const int pid = m4.w >> 6;
            valid[g] = lane < (m4.w & 63) && !epi.skip(pid);
            meta[g] = make_int2(m4.x + lane, valid[g] ? m4.y : 0);
            r[g] = m4.z + lane;
            if (valid[g]) pre[g] = epi.pre(r[g], pid);
#pragma unroll
            for (int a = 0; a < NACC; ++a) acc[g][a] = V(0);
            wmax = max(wmax, m4.y);
        }
    }
    for (int t0 = 0; t0 < wmax; t0 += B) {
        int ci[G][B];
        V va[G][B];
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const bool on = t0 + j < meta[g].y;
                const int q = meta[g].x + (t0 + j) * 32;
                ci[g][j] = on ? __ldcs(A.sell_ci + q) : 0;
                va[g][j] = on ? __ldcs(A.sell_val + q) : V(0);
            }
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int j = 0; j < B; ++j)
                if (t0 + j < meta[g].y) gather(ci[g][j], va[g][j], acc[g]);
    }
#pragma unroll
    for (int g = 0; g < G; ++g)
        if (valid[g]) epi(r[g], pre[g], acc[g]);
}

// --------------------------------------------------------------------------
// x-step
// --------------------------------------------------------------------------
template <typename V> struct GatherY {
    const V *ycomp;   // &UP[n].comp[cur] viewed as a stride-2 scalar array
    __device__ __forceinline__ void operator()(int i, V a, V (&acc)[1]) const {
        acc[0] = fma(a, __ldg(ycomp + 2 * (int64_t)i), acc[0]);
    }
};

template <typename V, bool KKT> struct EpiX {
    typedef typename Vec2<V>::T V2;
    struct Pre { V2 pr; V c, l, u; };
    static constexpr bool kRowOrder = true;
    const Prob<V> &P;
    V tau;
    int cur;
    Acc<V> &g2, &dres2, &lam, &cx;
    __device__ __forceinline__ bool skip(int) const { return false; }
    __device__ __forceinline__ Pre pre(int j, int) const {
        return Pre{P.UP[j], __ldg(P.c + j), __ldg(P.lo + j), __ldg(P.hi + j)};
    }
    __device__ __forceinline__ void operator()(int j, const Pre &in, const V (&s)[1]) {
        V2 pr = in.pr;
        const V x = comp<V>(pr, cur);
        const V cj = in.c, l = in.l, u = in.u;
        const V r = cj - s[0];
        V xh = x - tau * r;
        xh = xh < l ? l : (xh > u ? u : xh);
        if (cur) pr.x = xh; else pr.y = xh;
        P.UP[j] = pr;
        const V gx = xh - x;
        g2.add_sq(gx);
        if (KKT) {
            // lambda = P_Lambda(c - K'y), Lambda_j by finiteness of l_j, u_j (eq. lambda-case)
            const bool lf = isfinite(l), uf = isfinite(u);
            V lamj;
            if (!lf && !uf) lamj = V(0);
            else if (!lf) lamj = r < V(0) ? r : V(0);
            else if (!uf) lamj = r > V(0) ? r : V(0);
            else lamj = r;
            // residual in the caller's units: (c - K'y - lambda)_j = (scaled) / Dc_j
            V d = r - lamj;
            if (P.sc_x) d *= __ldg(P.sc_x + j);
            dres2.add_sq(d);
            if (lamj > V(0)) lam.add_prod(l, lamj);         // l' lambda+
            else if (lamj < V(0)) lam.add_prod(u, lamj);    // - u' lambda-
            cx.add_prod(cj, x);
        }
    }
};

template <typename V, bool KKT, int S = 0>
__global__ void __launch_bounds__(BLOCK) k_xstep(Prob<V> P, MethodParams mp, int mode) {
    constexpr TaskShape ts = task_shape(S);
    if (mode < MODE_EVAL && (P.st->done | P.st->error)) return;
    const int cur = (mode == MODE_INIT || !P.st->init_done) ? 0 : (int)(P.st->it & 1) ^ 1;
    __shared__ double sh[WARPS * 4];
    Acc<V> g2, dres2, lam, cx;
    GatherY<V> gat{reinterpret_cast<const V *>(P.UP + P.n) + cur};
    EpiX<V, KKT> epi{P, (V)mp.tau, cur, g2, dres2, lam, cx};
    const int warp = threadIdx.x >> 5;
    const int64_t ntask = P.KT.ntasks(ts.g);
    for (int64_t vb = blockIdx.x; vb * WARPS < ntask; vb += gridDim.x) {
        const int64_t t = vb * WARPS + warp;
        if (t < ntask) run_task<V, 1, ts.g, ts.ld>(P.KT, t, gat, epi);
    }
    if constexpr (KKT) {
        Acc<V> a4[4] = {g2, dres2, lam, cx};
        block_reduce_store<V, 4>(a4, sh, P.part1 + (int64_t)blockIdx.x * 4);
    } else {                                   // only ||g||^2 is used without KKT terms
        Acc<V> a1[1] = {g2};
        block_reduce_store<V, 1>(a1, sh, P.part1 + (int64_t)blockIdx.x * 4);
    }
}

// --------------------------------------------------------------------------
// y-step
// --------------------------------------------------------------------------
template <typename V, bool KKT> struct GatherXZ {
    typedef typename Vec2<V>::T V2;
    const V2 *UP;
    int cur;
    __device__ __forceinline__ void operator()(int j, V a, V (&acc)[KKT ? 2 : 1]) const {
        const V2 pr = __ldg(UP + j);
        const V x = cur ? pr.y : pr.x, xh = cur ? pr.x : pr.y;
        acc[0] = fma(a, V(2) * xh - x, acc[0]);
        if (KKT) acc[1] = fma(a, x, acc[1]);
    }
};

template <typename V, bool KKT> struct EpiY {
    typedef typename Vec2<V>::T V2;
    struct Pre { V2 pr; V q, l; };
    static constexpr bool kRowOrder = true;
    const Prob<V> &P;
    V sigma;
    int cur;
    Acc<V> &g2, &pres2, &qy;
    __device__ __forceinline__ bool skip(int) const { return false; }
    __device__ __forceinline__ Pre pre(int i, int) const {
        return Pre{P.UP[P.n + i], __ldg(P.q + i), __ldg(P.lo + P.n + i)};
    }
    __device__ __forceinline__ void operator()(int i, const Pre &in, const V (&t)[KKT ? 2 : 1]) {
        V2 pr = in.pr;
        const V y = comp<V>(pr, cur);
        const V qi = in.q, l = in.l;
        V yh = y + sigma * (qi - t[0]);
        yh = yh < l ? l : yh;                       // P_Y: y_i >= 0 on '>=' rows
        if (cur) pr.x = yh; else pr.y = yh;
        P.UP[P.n + i] = pr;
        g2.add_sq(yh - y);
        if (KKT) {
            V p = qi - t[1];                        // q - K x^k
            if (l == V(0) && p < V(0)) p = V(0);    // '>=' rows: only violation counts
            if (P.sc_y) p *= __ldg(P.sc_y + i);     // caller's units: (q - Kx)_i = (scaled) / Dr_i
            pres2.add_sq(p);
            qy.add_prod(qi, y);
        }
    }
};

// Final reduction after both half-steps (one block): ||g^k||, KKT of u^k,
// termination flag, safeguard decision of Alg. 2 / Alg. 3.  Reads the block
// partials of the x-step (part1, grid1 blocks) and the y-step (part2).
template <typename V>
__device__ void finalize_T(const Prob<V> &P, const MethodParams &mp, int mode, bool kkt) {
    __shared__ double sh[WARPS * 4];
    double a1[4] = {0, 0, 0, 0}, a2[3] = {0, 0, 0};
    if (kkt) {
        block_sum_columns<4>(P.part1, P.grid1, 4, a1, sh);
        block_sum_columns<3>(P.part2, P.grid2, 3, a2, sh);
    } else {                                   // only ||g||^2 without KKT terms
        double b1[1], b2[1];
        block_sum_columns<1>(P.part1, P.grid1, 4, b1, sh);
        block_sum_columns<1>(P.part2, P.grid2, 3, b2, sh);
        a1[0] = b1[0];
        a2[0] = b2[0];
    }
    if (threadIdx.x != 0) return;
    const double g2 = a1[0] + a2[0];
    const double dres2 = a1[1], lam = a1[2], cx = a1[3], pres2 = a2[1], qy = a2[2];
    DevState *st = P.st;
    const double gn = sqrt(g2);
    double out[6] = {0, 0, 0, 0, 0, 0};
    if (kkt) {
        const double dobj = qy + lam, pobj = cx;
        out[0] = sqrt(pres2) / (1.0 + mp.q_norm);
        out[1] = sqrt(dres2) / (1.0 + mp.c_norm);
        out[2] = fabs(dobj - pobj) / (1.0 + fabs(dobj) + fabs(pobj));
        out[3] = fmax(out[0], fmax(out[1], out[2]));
        out[4] = pobj;
        out[5] = dobj;
    }
    if (mode == MODE_EVAL) {
        for (int k = 0; k < 6; ++k) st->kkt[k] = out[k];
        st->kkt_valid = 1;
        return;
    }
    if (!isfinite(gn) || (kkt && !isfinite(out[3]))) { st->error = 1; return; }
    st->gnorm_prev = mode == MODE_INIT ? NAN : st->gnorm;
    st->gnorm = gn;
    if (mode == MODE_INIT) { st->g0 = gn; return; }
    const int64_t it = st->it;
    if (it < P.tr.cap) P.tr.gnorm[it] = gn;
    if (kkt) {
        for (int k = 0; k < 6; ++k) st->kkt[k] = out[k];
        st->kkt_valid = 1;
        if (it < P.tr.cap) P.tr.kkt[it] = out[3];
        if (out[3] <= mp.tol) { st->done = 1; return; }
    }
    bool want = false;
    if (mp.method != 0 && mp.mem > 0) {
        const double thr = mp.D * st->g0 * safeguard_factor(st, mp.c_div, mp.eps);
        want = gn <= thr;
    }
    st->want_aa = want ? 1 : 0;
}

template <typename V, bool KKT, int S = 0>
__global__ void __launch_bounds__(BLOCK) k_ystep(Prob<V> P, MethodParams mp, int mode) {
    constexpr TaskShape ts = task_shape(S);
    if (mode < MODE_EVAL && (P.st->done | P.st->error)) return;
    const int cur = (mode == MODE_INIT || !P.st->init_done) ? 0 : (int)(P.st->it & 1) ^ 1;
    __shared__ double sh[WARPS * 3];
    Acc<V> g2, pres2, qy;
    GatherXZ<V, KKT> gat{P.UP, cur};
    EpiY<V, KKT> epi{P, (V)mp.sigma, cur, g2, pres2, qy};
    const int warp = threadIdx.x >> 5;
    const int64_t ntask = P.K.ntasks(ts.g);
    for (int64_t vb = blockIdx.x; vb * WARPS < ntask; vb += gridDim.x) {
        const int64_t t = vb * WARPS + warp;
        if (t < ntask) run_task<V, KKT ? 2 : 1, ts.g, ts.ld>(P.K, t, gat, epi);
    }
    if (mode == MODE_TUNE) return;
    if constexpr (KKT) {
        Acc<V> a3[3] = {g2, pres2, qy};
        block_reduce_store<V, 3>(a3, sh, P.part2 + (int64_t)blockIdx.x * 3);
    } else {
        Acc<V> a1[1] = {g2};
        block_reduce_store<V, 1>(a1, sh, P.part2 + (int64_t)blockIdx.x * 3);
    }
}

// The final reduction after both half-steps, one block of its own: a
// last-block test in the y-step would have its ~900 co-resident blocks, which
// finish together, contend on one counter at the kernel's end.
template <typename V>
__global__ void __launch_bounds__(BLOCK) k_finalize(Prob<V> P, MethodParams mp, int mode, int kkt) {
    if (mode < MODE_EVAL && (P.st->done | P.st->error)) return;   // as the half-steps
    finalize_T<V>(P, mp, mode, kkt != 0);
}

// --------------------------------------------------------------------------
// Plain SpMV for the power iteration on K'K (Sec. 5.1 step-size rule).
// --------------------------------------------------------------------------
template <typename V> struct GatherPlain {
    const V *x;
    __device__ __forceinline__ void operator()(int j, V a, V (&acc)[1]) const {
        acc[0] = fma(a, __ldg(x + j), acc[0]);
    }
};
template <typename V, bool RowOrder> struct EpiStore {
    struct Pre {};
    static constexpr bool kRowOrder = RowOrder;
    V *y;
    Acc<V> &n2;
    __device__ __forceinline__ bool skip(int) const { return false; }
    __device__ __forceinline__ Pre pre(int, int) const { return Pre{}; }
    __device__ __forceinline__ void operator()(int r, const Pre &, const V (&s)[1]) {
        y[r] = s[0];
        n2.add_sq(s[0]);
    }
};

template <typename V, bool RowOrder = true>
__global__ void __launch_bounds__(BLOCK) k_spmv_plain(CSRView<V> A, const V *x, V *y, double *part) {
    __shared__ double sh[WARPS];
    Acc<V> n2;
    GatherPlain<V> gat{x};
    EpiStore<V, RowOrder> epi{y, n2};
    const int warp = threadIdx.x >> 5;
    const int64_t ntask = A.ntasks();
    for (int64_t vb = blockIdx.x; vb * WARPS < ntask; vb += gridDim.x) {
        const int64_t t = vb * WARPS + warp;
        if (t < ntask) run_task<V, 1>(A, t, gat, epi);
    }
    Acc<V> a1[1] = {n2};
    block_reduce_store<V, 1>(a1, sh, part + blockIdx.x);
}

template <typename V>
__global__ void k_scale(V *x, int64_t n, const double *part, int nb) {
    __shared__ double sh[BLOCK];
    const double s = block_sum_partials(part, nb, 1, 0, sh);
    const V f = (V)(s > 0 ? 1.0 / sqrt(s) : 0.0);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] *= f;
}

}  // namespace aap
