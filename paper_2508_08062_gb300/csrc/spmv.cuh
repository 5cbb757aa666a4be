// Fused PDHG half-steps (Sec. 3, eq. pdhg) on row-sliced CSR matrices.
//
// Both K and K' are stored as CSR with rows renumbered longest-first.  Rows are
// grouped in segments of equal "lanes per row" (lpr = 32, 16, ..., 1): a warp
// task covers 32 / lpr consecutive rows, each row read by lpr lanes with
// coalesced loads of its values and indices.  Rows longer than 32 * 32
// entries are split into LONG_CHUNK-entry chunks, one warp task each; the warp
// that finishes the last chunk of a row sums the chunk partials in chunk order
// (deterministic) and runs the row epilogue.
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
// into the NACC per-lane partial sums; epi(row, acc) runs once per row on one
// lane with the row's complete sums.
template <typename V, int NACC, class Gather, class Epi>
__device__ __forceinline__ void run_task(const CSRView<V> &A, int64_t t, Gather &gather, Epi &epi) {
    const int lane = threadIdx.x & 31;
    const SegTable &S = A.seg;
    int s = 0;
#pragma unroll 1
    while (s + 1 < S.nseg && t >= S.task0[s + 1]) ++s;
    const int64_t lt = t - S.task0[s];
    const int lpr = S.lpr[s];
    V acc[NACC];
#pragma unroll
    for (int a = 0; a < NACC; ++a) acc[a] = V(0);

    if (lpr == 0) {                                   // chunk of a split row
        const int chunk = (int)lt;
        const int r = __ldg(S.chunk_row + chunk);
        const int c0 = __ldg(S.row_chunk0 + r);
        const int nch = __ldg(S.row_chunk0 + r + 1) - c0;
        const int k0 = __ldg(A.rp + r) + (chunk - c0) * LONG_CHUNK;
        const int k1 = min(k0 + LONG_CHUNK, __ldg(A.rp + r + 1));
#pragma unroll 4
        for (int k = k0 + lane; k < k1; k += 32) gather(__ldg(A.ci + k), __ldg(A.val + k), acc);
#pragma unroll
        for (int a = 0; a < NACC; ++a)
#pragma unroll
            for (int o = 16; o; o >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
        int last = 0;
        if (lane == 0) {
#pragma unroll
            for (int a = 0; a < NACC; ++a) A.chunk_part[(int64_t)chunk * 2 + a] = acc[a];
            __threadfence();
            last = (atomicAdd(A.chunk_cnt + r, 1u) == (unsigned)(nch - 1));
        }
        last = __shfl_sync(0xffffffffu, last, 0);
        if (last && lane == 0) {
            __threadfence();
            V tot[NACC];
#pragma unroll
            for (int a = 0; a < NACC; ++a) tot[a] = V(0);
            for (int c = c0; c < c0 + nch; ++c)
#pragma unroll
                for (int a = 0; a < NACC; ++a) tot[a] += __ldcg(A.chunk_part + (int64_t)c * 2 + a);
            A.chunk_cnt[r] = 0u;
            epi(r, tot);
        }
        return;
    }

    const int rpw = 32 / lpr;
    const int r = S.row0[s] + (int)(lt * rpw) + lane / lpr;
    const int sub = lane & (lpr - 1);
    const bool valid = r < S.row1[s];
    if (valid) {
        const int k0 = __ldg(A.rp + r), k1 = __ldg(A.rp + r + 1);
#pragma unroll 4
        for (int k = k0 + sub; k < k1; k += lpr) gather(__ldg(A.ci + k), __ldg(A.val + k), acc);
    }
    for (int o = lpr >> 1; o; o >>= 1)
#pragma unroll
        for (int a = 0; a < NACC; ++a) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
    if (valid && sub == 0) epi(r, acc);
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
    const Prob<V> &P;
    V tau;
    int cur;
    Acc<V> &g2, &dres2, &lam, &cx;
    __device__ __forceinline__ void operator()(int j, const V (&s)[1]) {
        typedef typename Vec2<V>::T V2;
        V2 pr = P.UP[j];
        const V x = comp<V>(pr, cur);
        const V cj = __ldg(P.c + j), l = __ldg(P.lo + j), u = __ldg(P.hi + j);
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
            dres2.add_sq(r - lamj);
            if (lamj > V(0)) lam.add_prod(l, lamj);         // l' lambda+
            else if (lamj < V(0)) lam.add_prod(u, lamj);    // - u' lambda-
            cx.add_prod(cj, x);
        }
    }
};

template <typename V, bool KKT>
__global__ void __launch_bounds__(BLOCK) k_xstep(Prob<V> P, MethodParams mp, int mode) {
    if (mode != MODE_EVAL && (P.st->done | P.st->error)) return;
    const int cur = (mode == MODE_INIT || !P.st->init_done) ? 0 : (int)(P.st->it & 1) ^ 1;
    __shared__ double sh[WARPS * 4];
    Acc<V> g2, dres2, lam, cx;
    GatherY<V> gat{reinterpret_cast<const V *>(P.UP + P.n) + cur};
    EpiX<V, KKT> epi{P, (V)mp.tau, cur, g2, dres2, lam, cx};
    const int warp = threadIdx.x >> 5;
    const int64_t ntask = P.KT.seg.task0[P.KT.seg.nseg];
    for (int64_t vb = blockIdx.x; vb * WARPS < ntask; vb += gridDim.x) {
        const int64_t t = vb * WARPS + warp;
        if (t < ntask) run_task<V, 1>(P.KT, t, gat, epi);
    }
    Acc<V> a4[4] = {g2, dres2, lam, cx};
    block_reduce_store<V, 4>(a4, sh, P.part1 + (int64_t)blockIdx.x * 4);
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
    const Prob<V> &P;
    V sigma;
    int cur;
    Acc<V> &g2, &pres2, &qy;
    __device__ __forceinline__ void operator()(int i, const V (&t)[KKT ? 2 : 1]) {
        typedef typename Vec2<V>::T V2;
        V2 pr = P.UP[P.n + i];
        const V y = comp<V>(pr, cur);
        const V qi = __ldg(P.q + i), l = __ldg(P.lo + P.n + i);
        V yh = y + sigma * (qi - t[0]);
        yh = yh < l ? l : yh;                       // P_Y: y_i >= 0 on '>=' rows
        if (cur) pr.x = yh; else pr.y = yh;
        P.UP[P.n + i] = pr;
        g2.add_sq(yh - y);
        if (KKT) {
            V p = qi - t[1];                        // q - K x^k
            if (l == V(0) && p < V(0)) p = V(0);    // '>=' rows: only violation counts
            pres2.add_sq(p);
            qy.add_prod(qi, y);
        }
    }
};

// Final reduction after both half-steps (one block): ||g^k||, KKT of u^k,
// termination flag, safeguard decision of Alg. 2 / Alg. 3.
template <typename V>
__device__ void finalize_T(const Prob<V> &P, const MethodParams &mp, int mode, bool kkt) {
    __shared__ double sh[BLOCK];
    const double g2 = block_sum_partials(P.part1, P.grid1, 4, 0, sh) +
                      block_sum_partials(P.part2, P.grid2, 3, 0, sh);
    double dres2 = 0, lam = 0, cx = 0, pres2 = 0, qy = 0;
    if (kkt) {
        dres2 = block_sum_partials(P.part1, P.grid1, 4, 1, sh);
        lam = block_sum_partials(P.part1, P.grid1, 4, 2, sh);
        cx = block_sum_partials(P.part1, P.grid1, 4, 3, sh);
        pres2 = block_sum_partials(P.part2, P.grid2, 3, 1, sh);
        qy = block_sum_partials(P.part2, P.grid2, 3, 2, sh);
    }
    if (threadIdx.x != 0) return;
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
        const double thr = mp.D * st->g0 * pow((double)st->n_aa / mp.c_div + 1.0, -(1.0 + mp.eps));
        want = gn <= thr;
    }
    st->want_aa = want ? 1 : 0;
}

template <typename V, bool KKT>
__global__ void __launch_bounds__(BLOCK) k_ystep(Prob<V> P, MethodParams mp, int mode) {
    if (mode != MODE_EVAL && (P.st->done | P.st->error)) return;
    const int cur = (mode == MODE_INIT || !P.st->init_done) ? 0 : (int)(P.st->it & 1) ^ 1;
    __shared__ double sh[WARPS * 3];
    Acc<V> g2, pres2, qy;
    GatherXZ<V, KKT> gat{P.UP, cur};
    EpiY<V, KKT> epi{P, (V)mp.sigma, cur, g2, pres2, qy};
    const int warp = threadIdx.x >> 5;
    const int64_t ntask = P.K.seg.task0[P.K.seg.nseg];
    for (int64_t vb = blockIdx.x; vb * WARPS < ntask; vb += gridDim.x) {
        const int64_t t = vb * WARPS + warp;
        if (t < ntask) run_task<V, KKT ? 2 : 1>(P.K, t, gat, epi);
    }
    Acc<V> a3[3] = {g2, pres2, qy};
    block_reduce_store<V, 3>(a3, sh, P.part2 + (int64_t)blockIdx.x * 3);
    if (last_block(&P.st->cnt_spmv)) finalize_T<V>(P, mp, mode, KKT);
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
template <typename V> struct EpiStore {
    V *y;
    Acc<V> &n2;
    __device__ __forceinline__ void operator()(int r, const V (&s)[1]) {
        y[r] = s[0];
        n2.add_sq(s[0]);
    }
};

template <typename V>
__global__ void __launch_bounds__(BLOCK) k_spmv_plain(CSRView<V> A, const V *x, V *y, double *part) {
    __shared__ double sh[WARPS];
    Acc<V> n2;
    GatherPlain<V> gat{x};
    EpiStore<V> epi{y, n2};
    const int warp = threadIdx.x >> 5;
    const int64_t ntask = A.seg.task0[A.seg.nseg];
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
