// Shared device definitions of the AA-PDHG / FAA-PDHG CUDA path (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace aap {

constexpr int MAXM = 32;            // largest Anderson memory m_A
constexpr int NSLOT = MAXM + 1;     // ring slots: m_A columns + one slot for the next du
constexpr int BLOCK = 256;          // threads per block of the streaming kernels
constexpr int WARPS = BLOCK / 32;
constexpr int LONG_CHUNK = 1024;    // default entries per warp task of a long row
constexpr int SELL_MAX = 32;        // default: rows up to this length go to SELL-32 slices
constexpr int LOADS = 8;            // independent loads a lane keeps in flight
constexpr int SLICES_PER_TASK = 2;  // SELL slices one warp reads in lockstep

// Task shapes the SpMV kernels are compiled for: SELL slices per warp task and
// loads a lane keeps in flight.  The runtimes time every shape of the two
// half-step kernels on the actual matrices and keep the fastest (autotuning).
// All shapes sum every row in the same order, so the choice never changes a
// result.  Shape 0 is the default.
struct TaskShape {
    int g, ld;
};
constexpr int NSHAPE = 5;
__host__ __device__ constexpr TaskShape task_shape(int s) {
    return s == 1 ? TaskShape{1, 8}
         : s == 2 ? TaskShape{4, 8}
         : s == 3 ? TaskShape{1, 16}
         : s == 4 ? TaskShape{2, 16}
                  : TaskShape{SLICES_PER_TASK, LOADS};
}

// ---------------------------------------------------------------------------
// Accumulators.  FP64 mode: plain double.  Mixed mode: a float pair (hi, lo)
// fed with error-free transformations (exact product via fma, TwoSum), so a
// per-thread / per-warp partial carries about 44 significant bits, i.e. the
// accuracy of an FP64 accumulator over the same terms, while every operation
// runs on the FP32 pipes (the FP64 rate of this part is 1/64 of FP32).  The
// pair is rounded into a double once per warp and summed in FP64 from there.
// ---------------------------------------------------------------------------
template <typename V> struct Acc;

template <> struct Acc<double> {
    double s;
    __device__ __forceinline__ Acc() : s(0.0) {}
    __device__ __forceinline__ void add(double a) { s += a; }
    __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ void add_sq(double a) { s = fma(a, a, s); }
    __device__ __forceinline__ void warp_allreduce() {
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    __device__ __forceinline__ double value() const { return s; }
    // a warp's partial parked in shared memory, read back as value() would give it
    typedef double Packed;
    __device__ __forceinline__ Packed pack() const { return s; }
    static __device__ __forceinline__ double unpack(Packed p) { return p; }
};

template <> struct Acc<float> {
    float hi, lo;
    __device__ __forceinline__ Acc() : hi(0.f), lo(0.f) {}
    // TwoSum: hi + a = s + e exactly
    __device__ __forceinline__ void add(float a) {
        float s = __fadd_rn(hi, a);
        float bb = __fsub_rn(s, hi);
        float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(a, bb));
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ void add_prod(float a, float b) {
        float p = __fmul_rn(a, b);
        float e = __fmaf_rn(a, b, -p);      // a*b = p + e exactly
        add(p);
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ void add_sq(float a) { add_prod(a, a); }
    __device__ __forceinline__ void warp_allreduce() {
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
            float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
            add(h2);
            lo = __fadd_rn(lo, l2);
        }
    }
    __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
    // a warp's partial parked in shared memory as the float pair: the FP64
    // conversion is left to the one lane per column that sums the warps
    typedef float2 Packed;
    __device__ __forceinline__ Packed pack() const { return make_float2(hi, lo); }
    static __device__ __forceinline__ double unpack(Packed p) { return (double)p.x + (double)p.y; }
};

template <typename V> struct Vec2;
template <> struct Vec2<float> { typedef float2 T; };
template <> struct Vec2<double> { typedef double2 T; };

// ---------------------------------------------------------------------------
// Device-resident run state.  Written only by the single block that finishes
// a reduction (last-block pattern) and read by the streaming kernels.
// ---------------------------------------------------------------------------
struct DevState {
    int64_t it;            // loop iterations done
    int64_t n_aa, n_pd;    // i^k, j^k of Alg. 2
    int64_t n_lsfail;      // AA steps rejected by a failed factorisation
    int32_t done;          // KKT <= tol reached at the current iterate
    int32_t error;         // non-zero: NaN/Inf met (iterate left unchanged)
    int32_t init_done;     // u^1 = T u^0 and g^0 formed
    int32_t want_aa;       // safeguard passed this iteration
    int32_t accept;        // AA step taken this iteration
    int32_t count;         // columns in the memory
    int32_t new_slot;      // slot receiving the column of this iteration
    int32_t free_slot;     // slot receiving u^{k+1} - u^k (next column's du)
    int32_t use_count;     // columns used by the accepted AA step
    int32_t list[NSLOT];   // memory columns, oldest first
    int32_t use[NSLOT];    // columns used by the step (slot ids, oldest first)
    double gamma[NSLOT];   // coefficient of used column t (parallel to use[])
    double G[NSLOT * NSLOT];  // Gram entries <dg_a, dg_b> by slot
    double rhs[NSLOT];     // <dg_s, g^k> by slot
    double en2[NSLOT];     // ||du_s||^2 by slot
    double g0;             // ||g^0||
    double gnorm;          // ||g^k||
    double gnorm_prev;     // ||g^{k-1}||
    int64_t thr_key;       // n_aa + 1 when thr_fac holds (i/c_div + 1)^-(1+eps) for i = n_aa
    double thr_fac;        // cached safeguard factor (FP64 pow is slow on this part)
    int32_t restart;       // primal weight update: this iteration restarts the memory
    double kkt[6];         // r_p, r_d, r_g, KKT, c'x, dual objective at u^k
    int32_t kkt_valid;
    uint32_t cnt_ring;     // last-block counter of the memory pass
    uint32_t cnt_norm;     // last-block counter of the norm kernels
    uint64_t stale;        // single LP: slots whose Gram entries with the other columns are pending
    uint32_t cnt_gram;     // last-block counter of the Gram pass
    double scratch[8];     // (kept by a reset: ||q||^2, ||c||^2 of the create)
};

// Safeguard factor (i^k / c_div + 1)^-(1+eps) of Alg. 2 (reading R3), cached
// per value of i^k = n_aa: it changes only when an AA step is accepted.
__device__ __forceinline__ double safeguard_factor(DevState *st, double c_div, double eps) {
    if (st->thr_key != st->n_aa + 1) {
        st->thr_fac = pow((double)st->n_aa / c_div + 1.0, -(1.0 + eps));
        st->thr_key = st->n_aa + 1;
    }
    return st->thr_fac;
}

// Method parameters (by value into the kernels).
struct MethodParams {
    int32_t method;        // 0 PDHG, 1 AA, 2 FAA
    int32_t mem;           // m_A
    double tau, sigma;
    double D, eps, eta, beta, c_s, kappa, c_div;
    int32_t faa_adaptive;
    double tol;
    int32_t kkt_every;
    double q_norm, c_norm; // ||q||_2, ||c||_2 (Remark on termination)
};

// Trace buffers (device); cap = 0 disables.
struct Trace {
    int64_t cap;
    int8_t *branch;
    double *gnorm;
    double *kkt;
    int32_t *mk;
};

// One sparse matrix (K or K') with rows renumbered longest first, in two parts:
//  - n_long rows longer than the layout's slice width limit (SELL_MAX by
//    default; "long rows", numbered by a long-row id): CSR, cut into chunks of
//    at most long_chunk entries, one warp task per chunk (a row with several
//    chunks is finished by the warp whose chunk arrives last);
//  - the other rows: SELL-32 slices of up to 32 consecutive rows stored
//    column by column (entry t of the rows contiguous), padded with zero
//    entries (column 0, value 0) to the slice's longest row; one warp task
//    per SLICES_PER_TASK slices, lane = row of each slice.
// Every chunk and slice names its rows and the problem they belong to, so one
// matrix may hold the block-diagonal K of a batch of LPs, its slices ordered
// by width across all problems (a single LP is problem 0).
// The full CSR (rp, ci, val) is kept for the set-up kernels.
template <typename V> struct CSRView {
    int32_t rows;
    const int32_t *rp;
    const int32_t *ci;
    const V *val;
    int32_t n_long, n_chunks, n_slices;
    const int4 *chunk_meta;       // chunk -> (row, long-row id, problem, 0)
    const int32_t *row_chunk0;    // long-row id -> first chunk (n_long + 1 entries)
    const int4 *slice_meta;       // slice -> (offset of its first entry in sell_*, width,
                                  //           first row, rows | problem << 6)
    const int32_t *sell_ci;
    const V *sell_val;
    V *chunk_part;                // n_chunks * 2 partial sums of split rows
    uint32_t *chunk_cnt;          // arrival counters by long-row id (self-resetting)
    int32_t long_chunk;           // entries per warp task of a long row (the layout's)
    __host__ __device__ int64_t ntasks(int g = SLICES_PER_TASK) const {
        return (int64_t)n_chunks + (n_slices + g - 1) / g;
    }
};

// Everything a kernel needs about the problem and the iterate buffers.
template <typename V> struct Prob {
    typedef typename Vec2<V>::T V2;
    int32_t m, n;
    int64_t N, Npad;
    CSRView<V> KT;                // rows = variables (internal order), cols = rows of K
    CSRView<V> K;                 // rows = constraints (internal order)
    V2 *UP;                       // (u-hat, u) pairs, x part [0, n), y part [n, N)
    const V *c;                   // n
    const V *q;                   // m
    const V *lo, *hi;             // N: bounds of X, and (0 or -inf, +inf) for Y
    const V *dh;                  // N: D-hat
    V *g;                         // N: g^{k-1} / g^k
    V *DG, *W;                    // NSLOT * Npad rings: dg and du + beta D dg
    const V *sc_x, *sc_y;         // 1 / Dc (n) and 1 / Dr (m) when the LP is scaled, else null
    double *part1, *part2, *part3;// block partials of the x-step, y-step, memory pass
    int32_t grid1, grid2, grid3;  // grids of those kernels (fixed: deterministic sums)
    double *part4;                // single LP: block partials of the Gram pass
    int32_t grid4;
    DevState *st;
    Trace tr;
};

// Iterate storage: UP[e] = (comp0, comp1); comp[cur] is u^k, comp[1 - cur]
// receives T(u^k).  The roles swap every iteration, so a PDHG step never copies.
template <typename V>
__device__ __forceinline__ V comp(const typename Vec2<V>::T &p, int c) { return c ? p.y : p.x; }

// W consecutive elements, loaded / stored as one 16-byte vector when W*sizeof(V) == 16.
template <typename V, int W> struct alignas(sizeof(V) * W) Pack { V v[W]; };

template <typename V, int W>
__device__ __forceinline__ Pack<V, W> ld(const V *p) { return *reinterpret_cast<const Pack<V, W> *>(p); }

// Streaming (evict-first) load: data read once per iteration.
template <typename V, int W>
__device__ __forceinline__ Pack<V, W> ld_stream(const V *p) {
    Pack<V, W> r;
    if constexpr (W * sizeof(V) == 16) {
        if constexpr (sizeof(V) == 4) {
            const float4 t = __ldcs(reinterpret_cast<const float4 *>(p));
            r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
        } else {
            const double2 t = __ldcs(reinterpret_cast<const double2 *>(p));
            r.v[0] = t.x; r.v[1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < W; ++i) r.v[i] = __ldcs(p + i);
    }
    return r;
}

template <typename V, int W>
__device__ __forceinline__ void st(V *p, const Pack<V, W> &v) { *reinterpret_cast<Pack<V, W> *>(p) = v; }

// Kernel modes: forming u^1 = T u^0 and g^0, a loop iteration, a KKT
// evaluation of the current iterate that changes no run state, or a timing
// launch of a half-step (autotuning) that changes no run state either.
enum { MODE_INIT = 0, MODE_ITER = 1, MODE_EVAL = 2, MODE_TUNE = 3 };

// Block-wide sum of NV per-thread accumulators into FP64 (fixed order),
// written to out[0..NV) by thread 0 of the block.  `sh` holds WARPS * NV doubles.
template <typename V, int NV>
__device__ __forceinline__ void block_reduce_store(Acc<V> (&acc)[NV], double *sh, double *out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        acc[k].warp_allreduce();
        if (lane == 0) sh[warp * NV + k] = acc[k].value();
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < WARPS; ++w) s += sh[w * NV + threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// Last-block detection: every block calls after writing its partial; returns
// true in exactly one block (the last to arrive), which then owns the final
// reduction.  The counter resets itself.
__device__ __forceinline__ bool last_block(uint32_t *cnt) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t prev = atomicAdd(cnt, 1u);
        is_last = (prev == gridDim.x - 1);
        if (is_last) *cnt = 0u;
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// Fixed-order FP64 sums over `nb` blocks of columns [0, NC) of part[nb][stride]
// in one pass (one load round, warp shuffles, one shared-memory stage), by one
// block; out[k] is valid in thread 0 on return (the only thread that needs
// it: FP64 issue is scarce on this part, so the other warps skip the last
// stage).
template <int NC>
__device__ __forceinline__ void block_sum_columns(const double *part, int nb, int stride,
                                                  double (&out)[NC], double *sh) {
    double s[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) s[k] = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < NC; ++k) s[k] += __ldcg(part + (int64_t)b * stride + k);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
#pragma unroll
        for (int o = 16; o; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
        if (lane == 0) sh[warp * NC + k] = s[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            double t = 0.0;
            for (int w = 0; w < nw; ++w) t += sh[w * NC + k];
            out[k] = t;
        }
    }
    __syncthreads();
}

// Fixed-order FP64 sum over `nb` blocks of column k of part[nb][stride], by
// one block (all threads), result broadcast through shared memory.
__device__ __forceinline__ double block_sum_partials(const double *part, int nb, int stride,
                                                     int k, double *sh) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += __ldcg(part + (int64_t)b * stride + k);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

}  // namespace aap
