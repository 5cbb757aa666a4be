// Batched AA-PDHG / FAA-PDHG: many independent LPs advanced together.
//
// The batch is packed as one block-diagonal LP: K = diag(K_1, ..., K_P), the
// variables of all problems first (problem after problem), then their
// constraints, each problem's two ranges padded to multiples of 4 with inert
// elements (a variable fixed at 0 with zero cost, an empty '=' row with
// q = 0), which stay 0 and add nothing to any sum.  Each problem keeps the
// single-LP row order (longest first) and the single-LP slices, so every row
// of T(u) is computed exactly as for that LP alone; the slices of all
// problems are ordered by width across the batch.
//
// All problems share one iterate parity: UP[e].comp[cur] holds u^k of every
// problem, with cur the parity of the batch's iteration counter.  Everything
// else is per problem, in its own DevState: its step sizes, its iteration
// count, its Anderson memory (the same slot-major rings, restricted to its
// elements), its safeguard and solve, its KKT test and stop flag.  A problem
// whose state says "not started" forms u^1 = T u^0 and g^0 in the iteration
// in which it joins; a problem that has converged or failed is skipped by
// every kernel (its two iterate components are made equal when it stops, so
// the parity no longer matters to it).
//
// Kernels of one iteration (the half-steps reuse the single-LP task loop):
//   k_xstep_b / k_ystep_b  the PDHG half-steps with per-problem tau, sigma;
//                          on KKT iterations the KKT terms of u^k per element;
//   k_kkt_b                per-problem KKT of u^k (Remark on termination) and
//                          the stop test (KKT iterations only);
//   k_memory_b             per chunk of a problem's elements: the new memory
//                          column plus ||g^k||^2 (chunk partial sums);
//   k_gram_b               per problem (one warp): the fixed-order reduction of
//                          its chunk partials, its safeguard, the column
//                          appended (and, when the safeguard failed, the end
//                          of its iteration);
//   k_gram_cols_b, k_solve_b  the Gram pass and the m x m work of the problems
//                          whose safeguard passed (their AA attempts);
//   k_mix_b                the AA mix of the problems whose step was accepted.
#pragma once
#include "anderson.cuh"
#include "common.cuh"
#include "spmv.cuh"

namespace aap {

constexpr int BCHUNK = 8192;          // elements per chunk of a problem (multiple of 4)
constexpr int NBV = 5;                // chunk partial columns (the KKT terms; the memory pass uses 4)

template <typename V> struct BatchView {
    int32_t nprob;
    int64_t n_tot, m_tot;             // variables and constraints of all problems (padded)
    const double *tau, *sigma;        // per problem
    const V *tau_v, *sigma_v;         // the same in the iterate precision (no per-row conversion)
    DevState *stb;                    // per problem
    V *kterm;                         // KKT terms: 3 arrays over variables, then 2 over constraints
    int32_t nchunk;
    const int4 *chunk;                // chunk -> (problem, first element, length, 0: x part / 1: y part)
    const int32_t *pchunk0;           // problem -> first chunk (nprob + 1 entries)
    double *cpart;                    // nchunk * NBV chunk partials
    double *gpart;                    // nchunk * GRAM_MAXPAIRS Gram-pass partials (with a memory)
    uint32_t *pcnt;                   // per-problem arrival counters (self-resetting)
    const double *pnorm;              // per problem: ||q||, ||c|| of the caller's LP
    const double *ptol;               // per-problem tolerances, or null (one tolerance for all)
    int32_t pw_on;                    // primal weight update on: ||g^k|| also without a memory
};

__device__ __forceinline__ bool stopped(const DevState *s) { return (s->done | s->error) != 0; }

// Sum of p[c * stride] over chunks c0 <= c < c1 in chunk order (one thread),
// with the loads of 8 chunks issued before their adds.
__device__ __forceinline__ double ordered_chunk_sum(const double *p, int64_t stride, int c0, int c1) {
    double v = 0.0;
    for (int c = c0; c < c1; c += 8) {
        double t[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) t[j] = c + j < c1 ? __ldcg(p + (int64_t)(c + j) * stride) : 0.0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (c + j < c1) v += t[j];
    }
    return v;
}

// --------------------------------------------------------------------------
// Half-step epilogues (eq. pdhg per row, step sizes of the row's problem)
// --------------------------------------------------------------------------
template <typename V, bool KKT> struct EpiXB {
    typedef typename Vec2<V>::T V2;
    struct Pre { V2 pr; V c, l, u, tau; int keep; };
    static constexpr bool kRowOrder = false;
    const Prob<V> &P;
    const BatchView<V> &B;
    int cur, mode;
    __device__ __forceinline__ bool skip(int p) const {
        return mode != MODE_EVAL && stopped(B.stb + p);
    }
    __device__ __forceinline__ Pre pre(int j, int p) const {
        return Pre{P.UP[j], __ldg(P.c + j), __ldg(P.lo + j), __ldg(P.hi + j), __ldg(B.tau_v + p),
                   (int)stopped(B.stb + p)};
    }
    __device__ __forceinline__ void operator()(int j, const Pre &in, const V (&s)[1]) {
        V2 pr = in.pr;
        const V x = comp<V>(pr, cur);
        const V r = in.c - s[0];
        V xh = x;                                      // a stopped problem keeps its iterate
        if (!in.keep) {
            xh = x - in.tau * r;
            xh = xh < in.l ? in.l : (xh > in.u ? in.u : xh);
        }
        if (cur) pr.x = xh; else pr.y = xh;
        P.UP[j] = pr;
        if (KKT) {
            // lambda = P_Lambda(c - K'y) (eq. lambda-case), as in the single-LP epilogue
            const bool lf = isfinite(in.l), uf = isfinite(in.u);
            V lamj;
            if (!lf && !uf) lamj = V(0);
            else if (!lf) lamj = r < V(0) ? r : V(0);
            else if (!uf) lamj = r > V(0) ? r : V(0);
            else lamj = r;
            V d = r - lamj;
            if (P.sc_x) d *= __ldg(P.sc_x + j);
            V lt = V(0);
            if (lamj > V(0)) lt = in.l * lamj;
            else if (lamj < V(0)) lt = in.u * lamj;
            B.kterm[j] = d * d;
            B.kterm[B.n_tot + j] = lt;
            B.kterm[2 * B.n_tot + j] = in.c * x;
        }
    }
};

template <typename V, bool KKT> struct EpiYB {
    typedef typename Vec2<V>::T V2;
    struct Pre { V2 pr; V q, l, sigma; int keep; };
    static constexpr bool kRowOrder = false;
    const Prob<V> &P;
    const BatchView<V> &B;
    int cur, mode;
    __device__ __forceinline__ bool skip(int p) const {
        return mode != MODE_EVAL && stopped(B.stb + p);
    }
    __device__ __forceinline__ Pre pre(int i, int p) const {
        return Pre{P.UP[P.n + i], __ldg(P.q + i), __ldg(P.lo + P.n + i), __ldg(B.sigma_v + p),
                   (int)stopped(B.stb + p)};
    }
    __device__ __forceinline__ void operator()(int i, const Pre &in, const V (&t)[KKT ? 2 : 1]) {
        V2 pr = in.pr;
        const V y = comp<V>(pr, cur);
        V yh = y;
        if (!in.keep) {
            yh = y + in.sigma * (in.q - t[0]);
            yh = yh < in.l ? in.l : yh;
        }
        if (cur) pr.x = yh; else pr.y = yh;
        P.UP[P.n + i] = pr;
        if (KKT) {
            V p = in.q - t[1];
            if (in.l == V(0) && p < V(0)) p = V(0);
            if (P.sc_y) p *= __ldg(P.sc_y + i);
            B.kterm[3 * B.n_tot + i] = p * p;
            B.kterm[3 * B.n_tot + B.m_tot + i] = in.q * y;
        }
    }
};

template <typename V, bool KKT, int S = 0>
__global__ void __launch_bounds__(BLOCK) k_xstep_b(Prob<V> P, BatchView<V> B, int cur, int mode) {
    constexpr TaskShape ts = task_shape(S);
    GatherY<V> gat{reinterpret_cast<const V *>(P.UP + P.n) + cur};
    EpiXB<V, KKT> epi{P, B, cur, mode};
    const int warp = threadIdx.x >> 5;
    const int64_t ntask = P.KT.ntasks(ts.g);
    for (int64_t vb = blockIdx.x; vb * WARPS < ntask; vb += gridDim.x) {
        const int64_t t = vb * WARPS + warp;
        if (t < ntask) run_task<V, 1, ts.g, ts.ld>(P.KT, t, gat, epi);
    }
}

template <typename V, bool KKT, int S = 0>
__global__ void __launch_bounds__(BLOCK) k_ystep_b(Prob<V> P, BatchView<V> B, int cur, int mode) {
    constexpr TaskShape ts = task_shape(S);
    GatherXZ<V, KKT> gat{P.UP, cur};
    EpiYB<V, KKT> epi{P, B, cur, mode};
    const int warp = threadIdx.x >> 5;
    const int64_t ntask = P.K.ntasks(ts.g);
    for (int64_t vb = blockIdx.x; vb * WARPS < ntask; vb += gridDim.x) {
        const int64_t t = vb * WARPS + warp;
        if (t < ntask) run_task<V, KKT ? 2 : 1, ts.g, ts.ld>(P.K, t, gat, epi);
    }
}

// Arrival of one chunk of a problem with `nchunks` chunks: true in the block
// whose chunk arrives last (which then owns the problem's reduction).
__device__ __forceinline__ bool last_chunk(uint32_t *cnt, int nchunks) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        is_last = atomicAdd(cnt, 1u) == (unsigned)(nchunks - 1);
        if (is_last) *cnt = 0u;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// red[k] = sum over chunks [c0, c1) of column k of cpart, fixed order, for
// the columns set in `active`; one warp per column.
__device__ __forceinline__ void reduce_chunks(const double *cpart, int c0, int c1, int ncol,
                                              double *red, unsigned long long active) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = warp; k < ncol; k += WARPS) {
        if (!((active >> k) & 1ull)) continue;
        double v = 0.0;
        for (int c = c0 + lane; c < c1; c += 32) v += __ldcg(cpart + (int64_t)c * NBV + k);
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[k] = v;
    }
    __syncthreads();
}

// --------------------------------------------------------------------------
// Per-problem KKT of u^k (Remark on termination conditions) and, in mode
// ITER, the stop test KKT <= tol.  Grid: one block per chunk.
// --------------------------------------------------------------------------
template <typename V>
__global__ void __launch_bounds__(BLOCK) k_kkt_b(BatchView<V> B, double tol, int mode) {
    const int4 ch = B.chunk[blockIdx.x];
    const int p = ch.x;
    DevState *st = B.stb + p;
    if (mode != MODE_EVAL && (stopped(st) || !st->init_done)) return;
    Acc<V> a[5];
    const int64_t e1 = (int64_t)ch.y + ch.z;
    if (ch.w == 0) {
        for (int64_t j = ch.y + threadIdx.x; j < e1; j += BLOCK) {
            a[0].add(B.kterm[j]);
            a[1].add(B.kterm[B.n_tot + j]);
            a[2].add(B.kterm[2 * B.n_tot + j]);
        }
    } else {
        for (int64_t e = ch.y + threadIdx.x; e < e1; e += BLOCK) {
            const int64_t i = e - B.n_tot;
            a[3].add(B.kterm[3 * B.n_tot + i]);
            a[4].add(B.kterm[3 * B.n_tot + B.m_tot + i]);
        }
    }
    __shared__ double sh[WARPS * 5];
    block_reduce_store<V, 5>(a, sh, B.cpart + (int64_t)blockIdx.x * NBV);
    const int c0 = B.pchunk0[p], c1 = B.pchunk0[p + 1];
    if (!last_chunk(B.pcnt + p, c1 - c0)) return;
    __shared__ double red[NBV];
    reduce_chunks(B.cpart, c0, c1, 5, red, 0x1full);
    if (threadIdx.x != 0) return;
    const double dres2 = red[0], lam = red[1], cx = red[2], pres2 = red[3], qy = red[4];
    const double dobj = qy + lam, pobj = cx;
    double out[6];
    out[0] = sqrt(pres2) / (1.0 + B.pnorm[2 * p]);
    out[1] = sqrt(dres2) / (1.0 + B.pnorm[2 * p + 1]);
    out[2] = fabs(dobj - pobj) / (1.0 + fabs(dobj) + fabs(pobj));
    out[3] = fmax(out[0], fmax(out[1], out[2]));
    out[4] = pobj;
    out[5] = dobj;
    for (int k = 0; k < 6; ++k) st->kkt[k] = out[k];
    st->kkt_valid = 1;
    if (mode == MODE_ITER) {
        if (!isfinite(out[3])) st->error = 1;
        else if (out[3] <= (B.ptol ? B.ptol[p] : tol)) st->done = 1;
    }
}

// --------------------------------------------------------------------------
// Memory pass and ||g^k||^2, per chunk (one block each): a pure stream that
// writes the new memory column of the chunk's problem (dg, and du + beta
// D-hat dg) and the chunk's partial sums ||dg||^2, <dg, g^k>, ||du||^2 and
// ||g^k||^2 (columns 0-3 of cpart).  No old column is read: the new column's
// Gram entries are formed at the problem's next AA attempt (k_gram_cols_b),
// as in the single-LP solver.  A problem that stopped at this iteration's KKT
// test (done == 1) has its iterate copied into both components instead.
// --------------------------------------------------------------------------
template <typename V>
__global__ void __launch_bounds__(BLOCK) k_memory_b(Prob<V> P, BatchView<V> B, MethodParams mp, int cur) {
    constexpr int W = 16 / sizeof(V);
    typedef typename Vec2<V>::T V2;
    const int4 ch = B.chunk[blockIdx.x];
    const int p = ch.x;
    const DevState *st = B.stb + p;
    if (st->error || st->done == 2) return;
    const int64_t e0 = ch.y, e1 = (int64_t)ch.y + ch.z;
    if (st->done) {
        for (int64_t e = e0 + threadIdx.x; e < e1; e += BLOCK) {
            V2 pr = P.UP[e];
            if (cur) pr.x = pr.y; else pr.y = pr.x;
            P.UP[e] = pr;
        }
        return;
    }
    const bool init = !st->init_done;
    // the iteration of a primal weight update restarts the problem's memory:
    // a plain step, g^k kept as the previous residual, no column across it
    const bool restart = !init && st->restart;
    const int M = (mp.method == 0) ? 0 : mp.mem;
    if (M == 0 && !B.pw_on) return;
    const bool fresh = init || restart || M == 0;   // only g^k and ||g^k||^2
    __shared__ typename Acc<V>::Packed sh[WARPS * 4];
    // 0 ||dg||^2, 1 <dg, g>, 2 ||du||^2, 3 ||g||^2
    Acc<V> acc[4];
    const int64_t stride = (int64_t)BLOCK * W;
    if (fresh) {
        // g^k = T u^k - u^k (at the start: g^0 = u^1 - u^0, u^1 = T u^0 just
        // written into the other component)
        const V *UPs = reinterpret_cast<const V *>(P.UP);
        for (int64_t e = e0 + (int64_t)threadIdx.x * W; e < e1; e += stride) {
            const Pack<V, W> pa = ld<V, W>(UPs + 2 * e), pb = ld<V, W>(UPs + 2 * e + W);
            Pack<V, W> gk;
#pragma unroll
            for (int i = 0; i < W; ++i) {
                const int i0 = 2 * i, i1 = 2 * i + 1;
                const V a0 = i0 < W ? pa.v[i0 % W] : pb.v[i0 % W];
                const V a1 = i1 < W ? pa.v[i1 % W] : pb.v[i1 % W];
                gk.v[i] = (cur ? a0 : a1) - (cur ? a1 : a0);
                acc[3].add_sq(gk.v[i]);
            }
            aap::st<V, W>(P.g + e, gk);
        }
    } else {
        const int sn = st->free_slot;
        const bool prev_acc = st->accept != 0;
        V *DGn = P.DG + (int64_t)sn * P.Npad;
        V *Wn = P.W + (int64_t)sn * P.Npad;
        const V beta = (V)mp.beta;
        for (int64_t e = e0 + (int64_t)threadIdx.x * W; e < e1; e += stride)
            push_elems<V, W, true>(P, e, cur, prev_acc, beta, DGn, Wn, acc);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        acc[k].warp_allreduce();
        if (lane == 0) sh[warp * 4 + k] = acc[k].pack();
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int w = 0; w < WARPS; ++w) v += Acc<V>::unpack(sh[w * 4 + threadIdx.x]);
        B.cpart[(int64_t)blockIdx.x * NBV + threadIdx.x] = v;
    }
}

// --------------------------------------------------------------------------
// Per-problem reduction of the memory pass's chunk partials (fixed order),
// the safeguard of Alg. 2 / Alg. 3, and the new column appended to the
// problem's memory (the single-LP push).  A problem whose safeguard failed
// ends its iteration here (a PDHG step); one whose safeguard passed is
// finished by k_gram_cols_b and k_solve_b.  Grid: one warp per problem.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(32) k_gram_b(BatchView<float> Bf, BatchView<double> Bd, int fp64,
                                               MethodParams mp) {
    const int p = blockIdx.x;
    DevState *st = fp64 ? Bd.stb + p : Bf.stb + p;
    const int32_t *pchunk0 = fp64 ? Bd.pchunk0 : Bf.pchunk0;
    const double *cpart = fp64 ? Bd.cpart : Bf.cpart;
    const int lane = threadIdx.x;
    if (st->error || st->done == 2) return;
    if (st->done) {                       // stopped at this iteration's KKT test: now frozen
        if (lane == 0) {
            st->done = 2;
            st->restart = 0;              // an update at the stop iteration is not applied
            st->want_aa = 0;
        }
        return;
    }
    const bool init = !st->init_done;
    const bool restart = !init && st->restart;       // primal weight update (R15)
    const int M = (mp.method == 0) ? 0 : mp.mem;
    const bool norm = M > 0 || (fp64 ? Bd.pw_on : Bf.pw_on);
    __shared__ double red[4];
    __shared__ SolveSmem sm;
    // lane k sums column k over the problem's chunks in chunk order: one
    // FP64 add per chunk and lane, no cross-lane tree (FP64 issue is the
    // scarce resource here)
    const int c0 = pchunk0[p], c1 = pchunk0[p + 1];
    const bool fresh = init || restart || M == 0;
    if (norm && lane < 4 && (!fresh || lane == 3)) {
        double v = 0.0;
        v = ordered_chunk_sum(cpart + lane, NBV, c0, c1);
        red[lane] = v;
    }
    __syncwarp();
    const double gn = norm ? sqrt(red[3]) : 0.0;
    if (init || restart) {
        if (lane == 0) {
            if (!isfinite(gn)) st->error = 1;
            st->gnorm_prev = init ? NAN : st->gnorm;
            st->gnorm = gn;
            if (init) st->g0 = gn;
            st->count = 0;
            st->stale = 0ull;
            st->want_aa = 0;
            st->new_slot = 0;
            st->free_slot = 0;
            st->accept = 0;   // u^1 = T u^0 (or the restart step) behaves as a PDHG step
            st->use_count = 0;
            if (init) {
                st->it = 0;
                st->init_done = 1;
            } else {
                st->n_pd += 1;
                st->restart = 0;
                st->it += 1;
            }
        }
        return;
    }
    if (!isfinite(gn)) {
        if (lane == 0) {
            st->error = 1;
            st->want_aa = 0;
        }
        return;
    }
    if (lane == 0) {                      // the safeguard on one lane
        bool want = false;
        if (mp.method != 0 && M > 0)
            want = gn <= mp.D * st->g0 * safeguard_factor(st, mp.c_div, mp.eps);
        st->gnorm_prev = st->gnorm;
        st->gnorm = gn;
        st->want_aa = want ? 1 : 0;
    }
    __syncwarp();
    const Trace none{0, nullptr, nullptr, nullptr, nullptr};
    push_finalize(st, mp, M, M > 0 ? st->free_slot : 0, red, sm, none);
}

// --------------------------------------------------------------------------
// The Gram pass of the problems whose safeguard passed, in two kernels (the
// single-LP k_gram's work, per problem):
//   k_gram_cols_b  one block per (list position a, chunk) of such a problem:
//                  the chunk's partial dot products of column a with its
//                  partners in gram_pair_list (the columns b > a of its pairs
//                  (a, b), then g^k for the right-hand side), into gpart at
//                  the pairs' list indices;
//   k_solve_b      per such problem (one warp): the pairs' sums over its
//                  chunks in chunk order, the Gram entries and right-hand
//                  side, then the solve of Alg. 2 or the filters and solve of
//                  Alg. 3 and the end of the iteration.
// The blocks of one chunk read its column a once each and the partners
// (mostly the newest column and g^k) through L2, so an attempt moves about
// the k + 1 vectors once.  A block takes its partners GRAM_PG at a time.
// Every sum depends on the problem's own data only.
// --------------------------------------------------------------------------
constexpr int GRAM_PG = 8;                      // partners per pass over the chunk

template <typename V>
__global__ void __launch_bounds__(BLOCK) k_gram_cols_b(Prob<V> P, BatchView<V> B) {
    constexpr int W = 16 / sizeof(V);
    // blocks of one chunk are adjacent (x = list position), so the partners
    // they share stay in L2
    const int chunk = blockIdx.y;
    const int4 ch = B.chunk[chunk];
    const DevState *st = B.stb + ch.x;
    if (stopped(st) || !st->init_done || !st->want_aa) return;
    const int a = blockIdx.x, k = st->count;
    if (a >= k) return;
    __shared__ int s_pidx[NSLOT];                  // list index of each partner's pair
    __shared__ const V *s_vec[NSLOT];              // partner vectors
    __shared__ const V *s_col;
    __shared__ int s_np;
    __shared__ typename Acc<V>::Packed sh[WARPS * GRAM_PG];
    if (threadIdx.x == 0) {
        int list[NSLOT];
        for (int t = 0; t < k; ++t) list[t] = st->list[t];
        const uint64_t stale = st->stale;
        // the pairs of gram_pair_list in its order: (a', b) row pairs, then (a', k)
        int idx = 0, np = 0;
        for (int a2 = 0; a2 < k; ++a2)
            for (int b = a2 + 1; b < k; ++b)
                if (((stale >> list[a2]) | (stale >> list[b])) & 1ull) {
                    if (a2 == a) {
                        s_pidx[np] = idx;
                        s_vec[np] = P.DG + (int64_t)list[b] * P.Npad;
                        ++np;
                    }
                    ++idx;
                }
        if (a + 1 < k) {
            s_pidx[np] = idx + a;
            s_vec[np] = P.g;
            ++np;
        }
        s_np = np;
        s_col = P.DG + (int64_t)list[a] * P.Npad;
    }
    __syncthreads();
    const int np = s_np;
    const V *col = s_col;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t e0 = ch.y, e1 = (int64_t)ch.y + ch.z;
    for (int j0 = 0; j0 < np; j0 += GRAM_PG) {
        Acc<V> acc[GRAM_PG];
        for (int64_t e = e0 + (int64_t)threadIdx.x * W; e < e1; e += (int64_t)BLOCK * W) {
            const Pack<V, W> x = ld<V, W>(col + e);
#pragma unroll
            for (int j = 0; j < GRAM_PG; ++j)
                if (j0 + j < np) {
                    const Pack<V, W> y = ld<V, W>(s_vec[j0 + j] + e);
#pragma unroll
                    for (int i = 0; i < W; ++i) acc[j].add_prod(x.v[i], y.v[i]);
                }
        }
#pragma unroll
        for (int j = 0; j < GRAM_PG; ++j) {
            acc[j].warp_allreduce();
            if (lane == 0) sh[warp * GRAM_PG + j] = acc[j].pack();
        }
        __syncthreads();
        if (threadIdx.x < GRAM_PG && j0 + threadIdx.x < np) {
            double v = 0.0;
            for (int w = 0; w < WARPS; ++w) v += Acc<V>::unpack(sh[w * GRAM_PG + threadIdx.x]);
            B.gpart[(int64_t)chunk * GRAM_MAXPAIRS + s_pidx[j0 + threadIdx.x]] = v;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(32) k_solve_b(BatchView<float> Bf, BatchView<double> Bd, int fp64,
                                                MethodParams mp) {
    const int p = blockIdx.x;
    DevState *st = fp64 ? Bd.stb + p : Bf.stb + p;
    if (stopped(st) || !st->init_done || !st->want_aa) return;
    const int32_t *pchunk0 = fp64 ? Bd.pchunk0 : Bf.pchunk0;
    const double *gpart = fp64 ? Bd.gpart : Bf.gpart;
    const int lane = threadIdx.x;
    __shared__ int s_list[NSLOT];
    __shared__ int16_t s_pa[GRAM_MAXPAIRS], s_pb[GRAM_MAXPAIRS];
    __shared__ double s_val[GRAM_MAXPAIRS];
    __shared__ int s_np;
    __shared__ SolveSmem sm;
    const int k = st->count;
    if (lane == 0) {
        for (int a = 0; a < k; ++a) s_list[a] = st->list[a];
        s_np = gram_pair_list(s_list, k, st->stale, s_pa, s_pb);
    }
    __syncwarp();
    const int np = s_np;
    const int c0 = pchunk0[p], c1 = pchunk0[p + 1];
    for (int pr = lane; pr < np; pr += 32) {           // chunk order
        double v = 0.0;
        v = ordered_chunk_sum(gpart + pr, GRAM_MAXPAIRS, c0, c1);
        s_val[pr] = v;
    }
    __syncwarp();
    gram_store(st, s_list, k, s_pa, s_pb, np, s_val);
    const Trace none{0, nullptr, nullptr, nullptr, nullptr};
    memory_solve_tail(st, mp, mp.mem, sm, none);
}

// --------------------------------------------------------------------------
// AA mix of the problems whose step was accepted.  Grid: one block per chunk.
// --------------------------------------------------------------------------
template <typename V, int MC>
__global__ void __launch_bounds__(BLOCK) k_mix_b(Prob<V> P, BatchView<V> B, MethodParams mp, int cur) {
    constexpr int W = 16 / sizeof(V);
    const int4 ch = B.chunk[blockIdx.x];
    const DevState *st = B.stb + ch.x;
    if (stopped(st) || !st->init_done || !st->accept) return;
    const int64_t e0 = ch.y, e1 = (int64_t)ch.y + ch.z;
    __shared__ V s_gam[MC];
    __shared__ int64_t s_off[MC];
    if (threadIdx.x < MC) {
        const bool on = threadIdx.x < st->use_count;
        s_gam[threadIdx.x] = on ? (V)st->gamma[threadIdx.x] : V(0);
        s_off[threadIdx.x] = (int64_t)(on ? st->use[threadIdx.x] : 0) * P.Npad;
    }
    __syncthreads();
    const int k = st->use_count;
    V *Wf = P.W + (int64_t)st->free_slot * P.Npad;
    const V beta = (V)mp.beta;
    for (int64_t e = e0 + (int64_t)threadIdx.x * W; e < e1; e += (int64_t)BLOCK * W)
        mix_elems<V, MC, W>(P, e, cur, beta, s_gam, s_off, k, Wf);
}

// --------------------------------------------------------------------------
// Primal weight update of every running problem at an iterate u^k with
// k = 0 mod U_P (Alg. "Primal weight update" and the Remark on its form;
// readings R13-R15), on the device so that an asynchronous launch needs no
// host round trip:
//   k_pw_delta_b   per chunk: sum of (u^k - snapshot)^2 (the chunk is all x
//                  or all y), the snapshot becomes u^k (copy_only: the start);
//   k_pw_apply_b   per problem (one thread; pw = gamma, omega, lowest KKT at
//                  an update point): Delta_x, Delta_y from its chunk
//                  sums in chunk order; when both exceed epsilon_zero the new
//                  omega, tau = gamma / omega, sigma = gamma omega, the blend
//                  weight alpha from rho_k of ||g^{k-1}||, ||g^{k-2}|| (R14)
//                  and the restart flag (R15);
//   k_dhat_blend_b per chunk of an updated problem: D-hat =
//                  (1 - alpha) diag(1/omega, omega) + alpha diag(D1/omega, D2 omega).
// --------------------------------------------------------------------------
struct PwParams {
    double theta, eps_zero, rho_min, alpha_dec, alpha_inc;
};

template <typename V>
__global__ void __launch_bounds__(BLOCK) k_pw_delta_b(const typename Vec2<V>::T *UP, V *snap, BatchView<V> B,
                                                      int cur, int copy_only, double *part) {
    const int4 ch = B.chunk[blockIdx.x];
    const bool run = copy_only || !stopped(B.stb + ch.x);
    Acc<V> a[1];
    if (run)
        for (int64_t e = ch.y + (int64_t)threadIdx.x; e < (int64_t)ch.y + ch.z; e += BLOCK) {
            const V u = comp<V>(UP[e], cur);
            if (!copy_only) a[0].add_sq(u - snap[e]);
            snap[e] = u;
        }
    if (copy_only) return;
    __shared__ double sh[WARPS];
    block_reduce_store<V, 1>(a, sh, part + blockIdx.x);
}

template <typename V>
__global__ void k_pw_apply_b(BatchView<V> B, const double *part, double *pw, double *alpha, int32_t *upd,
                             PwParams pp) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= B.nprob) return;
    DevState *st = B.stb + p;
    upd[p] = 0;
    if (stopped(st)) return;
    double dx = 0.0, dy = 0.0;
    for (int c = B.pchunk0[p]; c < B.pchunk0[p + 1]; ++c) {
        if (B.chunk[c].w == 0) dx += part[c];
        else dy += part[c];
    }
    dx = sqrt(dx);
    dy = sqrt(dy);
    // FP32 iterates: an update only while the problem still improves, i.e.
    // its last KKT test is below every one seen at its earlier update points
    // (at FP32's attainable accuracy Delta_x, Delta_y are rounding noise and
    // an omega driven by them drifts; the FP64 path applies every update)
    bool improving = true;
    if (sizeof(V) == 4 && st->kkt_valid) {
        const double kk = st->kkt[3];
        improving = kk < pw[3 * p + 2];
        pw[3 * p + 2] = fmin(pw[3 * p + 2], kk);
    }
    if (!(dx > pp.eps_zero && dy > pp.eps_zero) || !improving) return;   // omega unchanged, no restart
    const double gamma = pw[3 * p];
    const double omega = exp(pp.theta * log(dy / dx) + (1.0 - pp.theta) * log(pw[3 * p + 1]));
    pw[3 * p + 1] = omega;
    const double tau = gamma / omega, sigma = gamma * omega;
    const_cast<double *>(B.tau)[p] = tau;
    const_cast<double *>(B.sigma)[p] = sigma;
    const_cast<V *>(B.tau_v)[p] = (V)tau;
    const_cast<V *>(B.sigma_v)[p] = (V)sigma;
    const double r1 = st->gnorm, r2 = st->gnorm_prev;
    const double rho = isnan(r2) ? 0.0 : (r2 - r1) / fmax(r2, pp.eps_zero);
    alpha[p] = rho >= pp.rho_min ? pp.alpha_dec : pp.alpha_inc;
    st->restart = 1;
    upd[p] = 1;
}

template <typename V>
__global__ void __launch_bounds__(BLOCK) k_dhat_blend_b(V *dh, const V *base, BatchView<V> B, const double *pw,
                                                        const double *alpha, const int32_t *upd) {
    const int4 ch = B.chunk[blockIdx.x];
    if (!upd[ch.x]) return;
    const double omega = pw[3 * ch.x + 1], a = alpha[ch.x];
    for (int64_t e = ch.y + (int64_t)threadIdx.x; e < (int64_t)ch.y + ch.z; e += BLOCK) {
        const double b = (1.0 - a) + a * (double)base[e];
        dh[e] = (V)(ch.w == 0 ? b / omega : b * omega);
    }
}

// Per-problem status for the host: (iterations, AA steps, PDHG steps, done,
// error, started).
__global__ void k_batch_status(const DevState *stb, int nprob, int64_t *out) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nprob; p += gridDim.x * blockDim.x) {
        out[6 * p] = stb[p].it;
        out[6 * p + 1] = stb[p].n_aa;
        out[6 * p + 2] = stb[p].n_pd;
        out[6 * p + 3] = stb[p].done;
        out[6 * p + 4] = stb[p].error;
        out[6 * p + 5] = stb[p].init_done;
    }
}

// A new solve call re-tests every problem against its own tolerance.
__global__ void k_batch_clear_done(DevState *stb, int nprob) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nprob; p += gridDim.x * blockDim.x)
        stb[p].done = 0;
}

// Power iteration per problem: out[s] = ||v||^2 over segment [off[s], off[s+1])
// (one block per segment, fixed order), and v scaled by 1 / sqrt(out[s]) there.
template <typename V>
__global__ void __launch_bounds__(BLOCK) k_seg_sumsq(const V *v, const int64_t *off, double *out) {
    const int s = blockIdx.x;
    Acc<V> a[1];
    for (int64_t e = off[s] + threadIdx.x; e < off[s + 1]; e += BLOCK) a[0].add_sq(v[e]);
    __shared__ double sh[WARPS];
    block_reduce_store<V, 1>(a, sh, out + s);
}

template <typename V>
__global__ void __launch_bounds__(BLOCK) k_seg_scale(V *v, const int64_t *off, const double *ss) {
    const int s = blockIdx.x;
    const V f = (V)(ss[s] > 0 ? 1.0 / sqrt(ss[s]) : 0.0);
    for (int64_t e = off[s] + threadIdx.x; e < off[s + 1]; e += BLOCK) v[e] *= f;
}

}  // namespace aap
