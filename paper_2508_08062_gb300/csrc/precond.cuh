// Diagonal preconditioning of the LP on the device (the Sec. 5.2 set-up:
// Ruiz scaling for 10 iterations combined with the Pock-Chambolle technique).
//
// A pass computes, from the current scaled K, one factor per row and one per
// column, 1 / sqrt(norm) (Ruiz: largest |entry|; Pock-Chambolle, alpha = 1:
// sum of |entries|; an empty row or column keeps 1), and multiplies every
// stored copy of K (CSR and SELL slices) and of K' by them.  The products of
// the factors are Dr (rows) and Dc (columns); the solver then iterates on
// Dr K Dc, Dr q, Dc c and the bounds divided by Dc.
#pragma once
#include "common.cuh"

namespace aap {

// out[r] = max_k |A_rk| (sum = 0) or sum_k |A_rk| (sum = 1); one warp per row.
template <typename V>
__global__ void k_row_norm(CSRView<V> A, int sum, V *out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); r < A.rows;
         r += warps) {
        V acc = V(0);
        for (int k = A.rp[r] + lane; k < A.rp[r + 1]; k += 32) {
            const V a = fabs(A.val[k]);
            acc = sum ? acc + a : fmax(acc, a);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            const V b = __shfl_xor_sync(0xffffffffu, acc, o);
            acc = sum ? acc + b : fmax(acc, b);
        }
        if (lane == 0) out[r] = acc;
    }
}

// d <- 1 / sqrt(d) where d > 0, else 1.
template <typename V>
__global__ void k_factor(V *d, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        d[i] = d[i] > V(0) ? V(1) / sqrt(d[i]) : V(1);
}

// A_rk <- A_rk * drow[r] * dcol[col(k)] for the CSR copy (one warp per row)
// and for the SELL slices (one warp per slice, lane = row).
template <typename V>
__global__ void k_scale_matrix(CSRView<V> A, const V *drow, const V *dcol) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t w0 = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    V *val = const_cast<V *>(A.val);
    for (int64_t r = w0; r < A.rows; r += warps) {
        const V fr = drow[r];
        for (int k = A.rp[r] + lane; k < A.rp[r + 1]; k += 32) val[k] = val[k] * fr * dcol[A.ci[k]];
    }
    V *sv = const_cast<V *>(A.sell_val);
    for (int64_t s = w0; s < A.n_slices; s += warps) {
        const int4 meta = A.slice_meta[s];
        const int64_t r = meta.z + lane;
        if (lane >= (meta.w & 63)) continue;
        const V fr = drow[r];
        for (int t = 0; t < meta.y; ++t) {
            const int64_t q = (int64_t)meta.x + (int64_t)t * 32 + lane;
            sv[q] = sv[q] * fr * dcol[A.sell_ci[q]];    // padding entries are 0 and stay 0
        }
    }
}

// D-hat of the Remark on its construction (mode 1) or the identity (mode 0):
// per row of K' (a variable) and per row of K (a constraint),
// sqrt(max(max |entry|, 1e-10)).  One warp per row, lanes striding its entries.
template <typename V>
__global__ void k_dhat(CSRView<V> KT, CSRView<V> K, int32_t n, int32_t m, int mode, V *dh) {
    const int64_t N = (int64_t)n + m;
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t e = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); e < N; e += warps) {
        if (mode == 0) { if (lane == 0) dh[e] = V(1); continue; }
        const CSRView<V> &A = e < n ? KT : K;
        const int32_t r = (int32_t)(e < n ? e : e - n);
        double mx = 0.0;
        for (int32_t k = A.rp[r] + lane; k < A.rp[r + 1]; k += 32) mx = fmax(mx, fabs((double)A.val[k]));
#pragma unroll
        for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) dh[e] = (V)sqrt(fmax(mx, 1e-10));
    }
}

// The same D-hat for one LP in the half-steps' layout (rows longest first:
// rows 0 .. n_long - 1 are long CSR rows cut into chunks, slice q holds rows
// n_long + 32 q on).  k_dhat_sliced runs one warp task per chunk or per SELL
// slice: a chunk's warp folds its max |entry| into its row's entry of dh (an
// atomic max on the bit pattern, which orders non-negative floats as
// integers; those entries start at 0), a slice is reduced by one lane per row
// with coalesced loads and finished at once; k_dhat_long then finishes the
// long rows.  |entry| and max are exact in any precision and order, so the
// result equals k_dhat's.
__device__ __forceinline__ void atomic_max_nonneg(float *p, float v) {
    atomicMax(reinterpret_cast<unsigned int *>(p), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_nonneg(double *p, double v) {
    atomicMax(reinterpret_cast<unsigned long long *>(p), (unsigned long long)__double_as_longlong(v));
}

template <typename V>
__device__ __forceinline__ void dhat_task(const CSRView<V> &A, int64_t t, V *out) {
    const int lane = threadIdx.x & 31;
    V mx = V(0);
    if (t < A.n_chunks) {
        const int chunk = (int)t;
        const int r = __ldg(reinterpret_cast<const int *>(A.chunk_meta + chunk));   // long-row id = row
        const int c0 = __ldg(A.row_chunk0 + r);
        const int k0 = __ldg(A.rp + r) + (chunk - c0) * A.long_chunk;
        const int k1 = min(k0 + A.long_chunk, __ldg(A.rp + r + 1));
        for (int k = k0 + lane; k < k1; k += 32) mx = fmax(mx, fabs(A.val[k]));
#pragma unroll
        for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) atomic_max_nonneg(out + r, mx);
        return;
    }
    const int64_t q = t - A.n_chunks;
    const int64_t r = A.n_long + q * 32 + lane;
    if (r >= A.rows) return;
    const int4 meta = A.slice_meta[q];          // offset, width (padding entries are 0)
    for (int tt = 0; tt < meta.y; ++tt) mx = fmax(mx, fabs(A.sell_val[(int64_t)meta.x + (int64_t)tt * 32 + lane]));
    out[r] = (V)sqrt(fmax((double)mx, 1e-10));
}

template <typename V>
__global__ void k_dhat_sliced(CSRView<V> KT, CSRView<V> K, int32_t n, int mode, V *dh) {
    const int64_t tx = (int64_t)KT.n_chunks + KT.n_slices, ty = (int64_t)K.n_chunks + K.n_slices;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t w0 = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    if (mode == 0) {
        for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n + K.rows;
             e += (int64_t)gridDim.x * blockDim.x)
            dh[e] = V(1);
        return;
    }
    for (int64_t t = w0; t < tx + ty; t += warps) {
        if (t < tx) dhat_task(KT, t, dh);
        else dhat_task(K, t - tx, dh + n);
    }
}

// Long rows: dh = sqrt(max(max |entry|, 1e-10)) from the maxima k_dhat_sliced folded in.
template <typename V>
__global__ void k_dhat_long(int32_t lx, int32_t ly, int32_t n, V *dh) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)lx + ly;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e < lx ? e : n + (e - lx);
        dh[i] = (V)sqrt(fmax((double)dh[i], 1e-10));
    }
}

// Primal weight update (Alg. "Primal weight update"): ||x^k - x^{k-U_P}||^2
// and ||y^k - y^{k-U_P}||^2 against the snapshot (into st->scratch[2], [3] by
// the last block), and the snapshot <- u^k.  copy_only: the snapshot alone.
template <typename V>
__global__ void __launch_bounds__(BLOCK) k_pw_delta(const typename Vec2<V>::T *UP, V *snap, int64_t n,
                                                    int64_t N, int cur, int copy_only, double *part,
                                                    DevState *st) {
    Acc<V> a[2];
    for (int64_t e = blockIdx.x * (int64_t)BLOCK + threadIdx.x; e < N; e += (int64_t)gridDim.x * BLOCK) {
        const V u = comp<V>(UP[e], cur);
        if (!copy_only) a[e < n ? 0 : 1].add_sq(u - snap[e]);
        snap[e] = u;
    }
    if (copy_only) return;
    __shared__ double sh[WARPS * 2];
    block_reduce_store<V, 2>(a, sh, part + 2 * (int64_t)blockIdx.x);
    if (last_block(&st->cnt_norm) && threadIdx.x == 0) {
        double sx = 0.0, sy = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) {
            sx += __ldcg(part + 2 * b);
            sy += __ldcg(part + 2 * b + 1);
        }
        st->scratch[2] = sx;
        st->scratch[3] = sy;
    }
}

// D-hat re-blend of the Remark on the primal weight's form:
// (1 - alpha) diag(1/omega, omega) + alpha diag(D1/omega, D2 omega).
template <typename V>
__global__ void k_dhat_blend(V *dh, const V *base, int64_t n, int64_t N, double omega, double alpha) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N;
         e += (int64_t)gridDim.x * blockDim.x) {
        const double b = (1.0 - alpha) + alpha * (double)base[e];
        dh[e] = (V)(e < n ? b / omega : b * omega);
    }
}

// Elementwise helpers: a *= b, a /= b, out = 1 / b, a = v.
template <typename V>
__global__ void k_vmul(V *a, const V *b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] *= b[i];
}
template <typename V>
__global__ void k_vdiv(V *a, const V *b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] /= b[i];
}
template <typename V>
__global__ void k_vinv(V *out, const V *b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = V(1) / b[i];
}
template <typename V>
__global__ void k_fill(V *a, V v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}

}  // namespace aap
