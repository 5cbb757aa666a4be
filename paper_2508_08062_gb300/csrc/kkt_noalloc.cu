// aapdhg_kkt_noalloc: KKT residuals of a caller-given point for an LP held in
// caller-owned device memory, with no device allocation at all.
//
// Some callers cannot allocate device memory at the moment they need the
// residuals: latency-critical loops that must not hit the implicit device
// synchronisation of cudaMalloc / cudaFree, and programs whose device memory
// is entirely owned by another framework's pool or fixed budget, where a
// private allocation would fail or fragment that pool.  This entry point
// serves them: its only scratch (block partial sums and an arrival counter)
// is a file-scope __device__ array of fixed size that every GPU loading the
// library holds until the process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <mutex>
#include <stdint.h>

#include "../../include/aapdhg.h"

namespace {

constexpr int NA_BLOCK = 256;                    // threads per block
constexpr int NA_WARPS = NA_BLOCK / 32;
constexpr int NA_ROWS = 512;                     // rows per block (64 per warp)
constexpr int NA_VALS = 8;                       // partial sums per block
constexpr int NA_MAX_DEVICES = 64;

// Block partials [AAPDHG_NOALLOC_MAX_BLOCKS][NA_VALS], then the arrival counter.
static __device__ __align__(256) double g_noalloc_scratch[AAPDHG_NOALLOC_MAX_BLOCKS * NA_VALS + 32];

std::mutex g_setup_mu;
void *g_scratch_ptr[NA_MAX_DEVICES] = {nullptr};

// Device address of the scratch array for the current device, resolved once
// per device (the name is only a host-side stand-in for the device symbol).
// The cached address belongs to the device's primary context: after a
// cudaDeviceReset it may be stale, which the header states.
cudaError_t scratch_for_current_device(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
    }
    *out = (double *)g_scratch_ptr[dev];
    return cudaSuccess;
}

// One warp per row, lanes striding the row's entries; FP64 throughout.
__device__ double warp_row_dot(const int64_t *rp, const int32_t *ci, const double *val,
                               const double *v, int64_t r) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int64_t k = rp[r] + lane; k < rp[r + 1]; k += 32) s = fma(val[k], v[ci[k]], s);
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Blocks [0, bx) walk the variables (rows of K'), blocks [bx, bx + by) the
// constraints (rows of K).  Partials per block, in slot order:
//   0 ||c - K'y - lambda||^2   1 l'lambda+ - u'lambda-   2 c'x   3 ||c||^2
//   4 primal violation^2       5 q'y                     6 ||q||^2
// The last block to arrive sums all partials in block order and writes out6.
__global__ void __launch_bounds__(NA_BLOCK)
k_kkt_noalloc(int32_t m, int32_t n, int bx, int by, const int64_t *rp, const int32_t *ci,
              const double *val, const int64_t *trp, const int32_t *tci, const double *tval,
              const int8_t *sense, const double *q, const double *c, const double *lb,
              const double *ub, const double *x, const double *y, double *out6, double *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc[NA_VALS] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int b = blockIdx.x;
    if (b < bx) {
        const int64_t r0 = (int64_t)b * NA_ROWS;
        for (int64_t j = r0 + warp; j < r0 + NA_ROWS && j < n; j += NA_WARPS) {
            const double s = warp_row_dot(trp, tci, tval, y, j);
            if (lane == 0) {
                const double r = c[j] - s, l = lb[j], u = ub[j];
                const bool lf = isfinite(l), uf = isfinite(u);
                double lam;
                if (!lf && !uf) lam = 0.0;                 // Lambda_j = {0}
                else if (!lf) lam = r < 0.0 ? r : 0.0;     // R_-
                else if (!uf) lam = r > 0.0 ? r : 0.0;     // R_+
                else lam = r;                              // R
                acc[0] += (r - lam) * (r - lam);
                if (lam > 0.0) acc[1] += l * lam;
                else if (lam < 0.0) acc[1] += u * lam;
                acc[2] += c[j] * x[j];
                acc[3] += c[j] * c[j];
            }
        }
    } else {
        const int64_t r0 = (int64_t)(b - bx) * NA_ROWS;
        for (int64_t i = r0 + warp; i < r0 + NA_ROWS && i < m; i += NA_WARPS) {
            const double t = warp_row_dot(rp, ci, val, x, i);
            if (lane == 0) {
                double p = q[i] - t;
                if (sense[i] == AAPDHG_ROW_GE && p < 0.0) p = 0.0;
                acc[4] += p * p;
                acc[5] += q[i] * y[i];
                acc[6] += q[i] * q[i];
            }
        }
    }
    // block sum in warp order (fixed)
    __shared__ double sh[NA_WARPS][NA_VALS];
    __shared__ bool last;
    if (lane == 0)
        for (int k = 0; k < NA_VALS; ++k) sh[warp][k] = acc[k];
    __syncthreads();
    unsigned int *counter = reinterpret_cast<unsigned int *>(scratch + AAPDHG_NOALLOC_MAX_BLOCKS * NA_VALS);
    if (threadIdx.x < NA_VALS) {
        double s = 0.0;
        for (int w = 0; w < NA_WARPS; ++w) s += sh[w][threadIdx.x];
        scratch[(int64_t)b * NA_VALS + threadIdx.x] = s;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == (unsigned int)(bx + by - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < NA_VALS) {
        double s = 0.0;
        for (int blk = 0; blk < bx + by; ++blk) s += __ldcg(scratch + (int64_t)blk * NA_VALS + threadIdx.x);
        sh[0][threadIdx.x] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double dres2 = sh[0][0], lamt = sh[0][1], cx = sh[0][2], c2 = sh[0][3];
        const double pres2 = sh[0][4], qy = sh[0][5], q2 = sh[0][6];
        const double dobj = qy + lamt, pobj = cx;
        const double r_p = sqrt(pres2) / (1.0 + sqrt(q2));
        const double r_d = sqrt(dres2) / (1.0 + sqrt(c2));
        const double r_g = fabs(dobj - pobj) / (1.0 + fabs(dobj) + fabs(pobj));
        out6[0] = r_p;
        out6[1] = r_d;
        out6[2] = r_g;
        out6[3] = fmax(r_p, fmax(r_d, r_g));
        out6[4] = pobj;
        out6[5] = dobj;
        *counter = 0u;    // the next call starts from zero
    }
}

}  // namespace

extern "C" aapdhg_status aapdhg_kkt_noalloc(int32_t m, int32_t n, const int64_t *row_ptr,
                                            const int32_t *col_idx, const double *val,
                                            const int64_t *t_row_ptr, const int32_t *t_col_idx,
                                            const double *t_val, const int8_t *row_sense,
                                            const double *q, const double *c, const double *lb,
                                            const double *ub, const double *x, const double *y,
                                            double *out6, void *cuda_stream) {
    if (m < 0 || n < 1) return AAPDHG_ERR_INVALID;
    const int64_t bx = ((int64_t)n + NA_ROWS - 1) / NA_ROWS;
    const int64_t by = ((int64_t)m + NA_ROWS - 1) / NA_ROWS;
    if (bx + by > AAPDHG_NOALLOC_MAX_BLOCKS) return AAPDHG_ERR_INVALID;   // beyond the fixed scratch
    // K has entries only when m > 0 (with m = 0 every row of K' is empty too)
    if (!row_ptr || !t_row_ptr || !c || !lb || !ub || !x || !out6 ||
        (m > 0 && (!col_idx || !val || !t_col_idx || !t_val || !row_sense || !q || !y)))
        return AAPDHG_ERR_INVALID;
    double *scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return AAPDHG_ERR_CUDA;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the arrival counter must start at zero: clear it (no allocation)
    if (cudaMemsetAsync(scratch + AAPDHG_NOALLOC_MAX_BLOCKS * NA_VALS, 0, sizeof(unsigned int), s) !=
        cudaSuccess) {
        cudaGetLastError();
        return AAPDHG_ERR_CUDA;
    }
    k_kkt_noalloc<<<(unsigned int)(bx + by), NA_BLOCK, 0, s>>>(m, n, (int)bx, (int)by, row_ptr, col_idx,
                                                               val, t_row_ptr, t_col_idx, t_val,
                                                               row_sense, q, c, lb, ub, x, y, out6,
                                                               scratch);
    if (cudaGetLastError() != cudaSuccess) return AAPDHG_ERR_CUDA;
    return AAPDHG_OK;
}
