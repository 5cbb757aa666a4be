// Host runtime and C ABI of the GB300 AA-PDHG / FAA-PDHG solver.
//
// create():  validate the CSR of K = [G; A] (eq. LP-O), renumber rows of K and
//            of K' longest-first, build both matrices in two parts (rows
//            longer than 32 entries as CSR chunks of 1024 entries, the others
//            as SELL-32 slices), move everything to the device and form D-hat
//            and ||q||, ||c|| there.
// iterate(): launch the per-iteration kernel sequence in chunks on the
//            handle's stream; poll the device-side done / error flags once per
//            chunk.  All branch decisions (termination, safeguard, factorisation
//            failure, filters) are taken on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/aapdhg.h"
#include "anderson.cuh"
#include "common.cuh"
#include "host.h"
#include "precond.cuh"
#include "spmv.cuh"

using namespace aap;

namespace {

aapdhg_alloc_fn g_alloc = nullptr;
aapdhg_free_fn g_free = nullptr;
void *g_ctx = nullptr;
thread_local std::string g_create_err;

constexpr int CHUNK_ITERS = 64;   // iterations launched between two host polls
static_assert(NSHAPE == AAPDHG_TASK_SHAPES, "task shapes of the C ABI and the kernels differ");

}  // namespace

namespace aaph {

void *raw_alloc(size_t bytes) {
    void *p = nullptr;
    if (g_alloc) return g_alloc(bytes, g_ctx);
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void raw_free(void *p) {
    if (g_free) g_free(p, g_ctx);
    else cudaFree(p);
}

bool build_layout(const HostCSR &A, const std::vector<RowSeg> &segs, LayoutHost &L,
                  const LayoutParams &prm) {
    auto len = [&](int32_t r) { return A.rp[r + 1] - A.rp[r]; };
    struct Slice { int32_t row0, rows, pid, width; };
    std::vector<int32_t> long_rows, long_pid;
    std::vector<Slice> sl;
    for (const RowSeg &sg : segs) {
        int32_t r = sg.row0;
        const int32_t end = sg.row0 + sg.rows;
        for (; r < end && len(r) > prm.sell_max; ++r) {
            long_rows.push_back(r);
            long_pid.push_back(sg.pid);
        }
        for (; r < end; r += 32) sl.push_back({r, std::min(32, end - r), sg.pid, len(r)});
    }
    L.n_long = (int32_t)long_rows.size();
    L.long_chunk = prm.long_chunk;
    L.row_chunk0.assign(L.n_long + 1, 0);
    for (int32_t lr = 0; lr < L.n_long; ++lr) {
        const int32_t nch = (len(long_rows[lr]) + prm.long_chunk - 1) / prm.long_chunk;
        L.row_chunk0[lr + 1] = L.row_chunk0[lr] + nch;
        for (int32_t c = 0; c < nch; ++c) L.chunk_meta.push_back(make_int4(long_rows[lr], lr, long_pid[lr], 0));
    }
    L.n_chunks = L.row_chunk0[L.n_long];
    std::stable_sort(sl.begin(), sl.end(), [](const Slice &a, const Slice &b) { return a.width > b.width; });
    L.n_slices = (int32_t)sl.size();
    int64_t total = 0;
    for (const Slice &x : sl) total += 32 * (int64_t)x.width;
    if (total >= ((int64_t)1 << 31)) return false;
    L.slice_meta.resize(L.n_slices);
    L.sell_ci.assign(total, 0);
    L.sell_val.assign(total, 0.0);
    std::vector<int64_t> soff(L.n_slices + 1, 0);
    for (int32_t q = 0; q < L.n_slices; ++q) {
        const Slice &x = sl[q];
        L.slice_meta[q] = make_int4((int32_t)soff[q], x.width, x.row0, x.rows | (x.pid << 6));
        soff[q + 1] = soff[q] + 32 * (int64_t)x.width;
    }
    run_ranges(weight_cuts(soff.data(), L.n_slices, host_threads(total)), [&](int, int64_t lo, int64_t hi) {
        for (int64_t q = lo; q < hi; ++q) {
            const Slice &x = sl[q];
            for (int32_t lane = 0; lane < x.rows; ++lane) {
                const int32_t r = x.row0 + lane, lrn = len(r);
                for (int32_t t = 0; t < lrn; ++t) {
                    const int64_t k = soff[q] + (int64_t)t * 32 + lane;
                    L.sell_ci[k] = A.ci[A.rp[r] + t];
                    L.sell_val[k] = A.val[A.rp[r] + t];
                }
            }
        }
    });
    return true;
}

int host_threads(int64_t work) {
    if (work < ((int64_t)1 << 20)) return 1;
    const unsigned hw = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(hw, 16u));
}

std::vector<int64_t> even_cuts(int64_t n, int T) {
    std::vector<int64_t> cuts(T + 1);
    for (int t = 0; t <= T; ++t) cuts[t] = n * t / T;
    return cuts;
}

// Indices [0, N) by decreasing len, ties in index order: a counting sort, so
// the permutation a stable sort by decreasing length gives, in linear time.
static void order_by_length(const std::vector<int64_t> &len, std::vector<int32_t> &perm) {
    const int64_t N = (int64_t)len.size();
    int64_t maxl = 0;
    for (int64_t l : len) maxl = std::max(maxl, l);
    std::vector<int64_t> start(maxl + 2, 0);
    for (int64_t l : len) start[maxl - l + 1]++;
    for (int64_t b = 1; b <= maxl + 1; ++b) start[b] += start[b - 1];
    perm.resize(N);
    for (int64_t i = 0; i < N; ++i) perm[start[maxl - len[i]]++] = (int32_t)i;
}

void build_internal(int32_t m, int32_t n, const int64_t *rp, const int32_t *ci, const double *val,
                    std::vector<int32_t> &perm_x, std::vector<int32_t> &perm_y, HostCSR &K,
                    HostCSR &KT) {
    const int64_t Z = rp[m];
    const int TH = host_threads(Z);
    // per-thread column counters over runs of consecutive rows (at most 2^27
    // counters in all): the column degrees here, the transpose below
    const int TT = (int)std::max<int64_t>(1, std::min<int64_t>(TH, ((int64_t)1 << 27) / std::max<int32_t>(n, 1)));
    std::vector<std::vector<int32_t>> cnt(TT);
    std::vector<int64_t> rlen(m), clen(n);
    for (int32_t i = 0; i < m; ++i) rlen[i] = rp[i + 1] - rp[i];
    run_ranges(weight_cuts(rp, m, TT), [&](int t, int64_t lo, int64_t hi) {
        cnt[t].assign(n, 0);
        for (int64_t k = rp[lo]; k < rp[hi]; ++k) cnt[t][ci[k]]++;
    });
    run_ranges(even_cuts(n, TH), [&](int, int64_t lo, int64_t hi) {
        for (int64_t j = lo; j < hi; ++j) {
            int64_t d = 0;
            for (int t = 0; t < TT; ++t) d += cnt[t][j];
            clen[j] = d;
        }
    });
    order_by_length(rlen, perm_y);
    order_by_length(clen, perm_x);
    std::vector<int32_t> inv_x(n);
    for (int32_t j = 0; j < n; ++j) inv_x[perm_x[j]] = j;
    // K: internal row ii is the caller's row perm_y[ii], its columns in the
    // internal order, ascending (rows in parallel)
    K.rows = m;
    K.rp.assign(m + 1, 0);
    for (int32_t ii = 0; ii < m; ++ii) K.rp[ii + 1] = K.rp[ii] + (int32_t)rlen[perm_y[ii]];
    K.ci.resize(Z);
    K.val.resize(Z);
    run_ranges(weight_cuts(K.rp.data(), m, TH), [&](int, int64_t lo, int64_t hi) {
        std::vector<std::pair<int32_t, double>> tmp;
        for (int64_t ii = lo; ii < hi; ++ii) {
            const int32_t i = perm_y[ii];
            const int64_t L = rlen[i], src = rp[i];
            int32_t *oc = K.ci.data() + K.rp[ii];
            double *ov = K.val.data() + K.rp[ii];
            if (L <= 32) {                                  // insertion sort in place
                for (int64_t t = 0; t < L; ++t) {
                    const int32_t cc = inv_x[ci[src + t]];
                    const double vv = val[src + t];
                    int64_t u = t;
                    for (; u > 0 && oc[u - 1] > cc; --u) {
                        oc[u] = oc[u - 1];
                        ov[u] = ov[u - 1];
                    }
                    oc[u] = cc;
                    ov[u] = vv;
                }
            } else {
                tmp.resize(L);
                for (int64_t t = 0; t < L; ++t) tmp[t] = {inv_x[ci[src + t]], val[src + t]};
                std::sort(tmp.begin(), tmp.end(),
                          [](const std::pair<int32_t, double> &a, const std::pair<int32_t, double> &b) {
                              return a.first < b.first;
                          });
                for (int64_t t = 0; t < L; ++t) {
                    oc[t] = tmp[t].first;
                    ov[t] = tmp[t].second;
                }
            }
        }
    });
    // K' = K transposed.  Each thread counts the columns of a run of
    // consecutive rows, the counts become start positions, and each thread
    // scatters its rows in order: every K' row lists its rows ascending, as
    // one sequential pass would.
    KT.rows = n;
    KT.rp.assign(n + 1, 0);
    for (int32_t jj = 0; jj < n; ++jj) KT.rp[jj + 1] = KT.rp[jj] + (int32_t)clen[perm_x[jj]];
    KT.ci.resize(Z);
    KT.val.resize(Z);
    const std::vector<int64_t> rc = weight_cuts(K.rp.data(), m, TT);
    run_ranges(rc, [&](int t, int64_t lo, int64_t hi) {
        std::fill(cnt[t].begin(), cnt[t].end(), 0);
        for (int64_t p = K.rp[lo]; p < K.rp[hi]; ++p) cnt[t][K.ci[p]]++;
    });
    run_ranges(even_cuts(n, TH), [&](int, int64_t lo, int64_t hi) {
        for (int64_t jj = lo; jj < hi; ++jj) {
            int32_t off = KT.rp[jj];
            for (int t = 0; t < TT; ++t) {
                const int32_t c = cnt[t][jj];
                cnt[t][jj] = off;
                off += c;
            }
        }
    });
    run_ranges(rc, [&](int t, int64_t lo, int64_t hi) {
        int32_t *pos = cnt[t].data();
        for (int64_t ii = lo; ii < hi; ++ii)
            for (int32_t p = K.rp[ii]; p < K.rp[ii + 1]; ++p) {
                const int32_t q = pos[K.ci[p]]++;
                KT.ci[q] = (int32_t)ii;
                KT.val[q] = K.val[p];
            }
    });
}

std::string validate_lp(int32_t m, int32_t n, int64_t nnz, const int64_t *row_ptr,
                        const int32_t *col_idx, const double *val, const int8_t *row_sense,
                        const double *q, const double *c, const double *lb, const double *ub) {
    if (m < 0 || n < 1 || nnz < 0 || nnz >= ((int64_t)1 << 31)) return "need m >= 0, n >= 1, 0 <= nnz < 2^31";
    if (!row_ptr || (nnz > 0 && (!col_idx || !val)) || (m > 0 && (!row_sense || !q)) || !c || !lb || !ub)
        return "NULL input array";
    if (row_ptr[0] != 0 || row_ptr[m] != nnz) return "row_ptr[0] must be 0 and row_ptr[m] must be nnz";
    // the rows before the first one whose pointer decreases (or leaves
    // [0, nnz]) are read; each row's checks run in order, and the error
    // reported is that of the first failing row
    int32_t r_bad = m;
    for (int32_t i = 0; i < m; ++i)
        if (row_ptr[i + 1] < row_ptr[i] || row_ptr[i + 1] > nnz) {
            r_bad = i;
            break;
        }
    const int TH = host_threads(nnz);
    const int TT = (int)std::max<int64_t>(1, std::min<int64_t>(TH, ((int64_t)1 << 27) / n));   // marks
    const std::vector<int64_t> cuts = weight_cuts(row_ptr, r_bad, TT);
    std::vector<int32_t> bad_row(TT, INT32_MAX);
    std::vector<const char *> bad_msg(TT, nullptr);
    run_ranges(cuts, [&](int t, int64_t lo, int64_t hi) {
        std::vector<int32_t> mark(n, -1);
        for (int64_t i = lo; i < hi; ++i) {
            const char *msg = nullptr;
            if (row_sense[i] != AAPDHG_ROW_EQ && row_sense[i] != AAPDHG_ROW_GE) {
                msg = "row_sense must be 0 (=) or 1 (>=)";
            } else {
                for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                    const int32_t j = col_idx[k];
                    if (j < 0 || j >= n) { msg = "column index out of range"; break; }
                    if (mark[j] == (int32_t)i) { msg = "repeated column within a row"; break; }
                    mark[j] = (int32_t)i;
                }
            }
            if (msg) {
                bad_row[t] = (int32_t)i;
                bad_msg[t] = msg;
                return;
            }
        }
    });
    int tb = 0;
    for (int t = 1; t < TT; ++t)
        if (bad_row[t] < bad_row[tb]) tb = t;
    if (bad_msg[tb]) return bad_msg[tb];
    if (r_bad < m) return "row_ptr is not non-decreasing";
    std::vector<char> nonfinite(TH, 0);
    run_ranges(even_cuts(nnz, TH), [&](int t, int64_t lo, int64_t hi) {
        for (int64_t k = lo; k < hi; ++k)
            if (!std::isfinite(val[k])) {
                nonfinite[t] = 1;
                return;
            }
    });
    for (char f : nonfinite)
        if (f) return "non-finite value in K, q or c";
    for (int32_t i = 0; i < m; ++i)
        if (!std::isfinite(q[i])) return "non-finite value in K, q or c";
    for (int32_t j = 0; j < n; ++j)
        if (!std::isfinite(c[j])) return "non-finite value in K, q or c";
    for (int32_t j = 0; j < n; ++j) {
        if (std::isnan(lb[j]) || std::isnan(ub[j]) || lb[j] > ub[j] || lb[j] == INFINITY || ub[j] == -INFINITY)
            return "bounds must satisfy lb <= ub, lb < +inf, ub > -inf";
    }
    return "";
}

}  // namespace aaph

using namespace aaph;

struct DevAlloc {
    void *p;
    size_t bytes;
};

struct aapdhg_s {
    int32_t m = 0, n = 0;
    int64_t nnz = 0, N = 0, Npad = 0;
    int32_t prec = AAPDHG_MIXED;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, sm_count = 0;
    aapdhg_status sticky = AAPDHG_OK;
    std::string err;
    std::vector<DevAlloc> allocs;
    int64_t bytes = 0;

    std::vector<int32_t> perm_x, perm_y;   // internal -> caller order
    std::vector<double> lo_x, hi_x;        // caller order bounds (projection of a start)
    std::vector<int8_t> sense;             // caller order
    std::vector<double> x0, y0;            // caller order start (projected)

    Prob<float> pf{};
    Prob<double> pd{};
    MethodParams mp{};
    bool have_steps = false;
    bool rings_ok = false;
    int32_t ring_mem = -1;                 // m_A the rings were sized for
    int32_t grid5 = 1;
    DevState *st = nullptr;
    DevState *st_host = nullptr;           // pinned mirror
    // trace
    int64_t tr_cap = 0;
    // kernel instrumentation (CUDA events on the handle's stream)
    bool prof_on = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_kind;
    double prof_ms[5] = {0, 0, 0, 0, 0};
    int64_t prof_n[5] = {0, 0, 0, 0, 0};
    int64_t launches = 0;
    // CUDA graphs of full chunks, keyed by the KKT phase of the chunk's first
    // iteration; invalidated whenever kernel parameters change
    cudaStream_t cap_stream = nullptr;
    struct GraphEntry {
        cudaGraphExec_t exec;
        int64_t phase;
        int32_t kkt_every;
        double tol;
        int64_t kernels;               // kernel launches in the captured chunk
    };
    std::vector<GraphEntry> graphs;
    bool use_graphs = true;
    // task shapes of the two half-step kernels (autotuned at the first iterate)
    int32_t shape_x = 0, shape_y = 0;
    bool tuned = false, autotune = true;
    // time limit of a run (the paper's one-hour cap); 0: none
    double time_limit = 0.0, time_used = 0.0;
    // layouts of K' and K (slice width limit, long-row chunk) and the device
    // allocations of their layout parts, by matrix (0: K', 1: K)
    LayoutParams lay[2];
    std::vector<void *> lay_ptrs[2];
    double lay_us[2 * AAPDHG_LAYOUT_CANDIDATES] = {};
    int32_t gridx[NSHAPE] = {}, gridy[NSHAPE] = {};
    double tune_us[2 * NSHAPE] = {};
    // primal weight update (off when pw_period = 0)
    int64_t pw_period = 0;
    double pw_theta = 0.5, pw_eps = 1e-10, pw_rho_min = 0.1, pw_alpha_dec = 0.1, pw_alpha_inc = 0.9;
    int32_t pw_dhat = 1;
    double pw_gamma = 0.0, pw_omega = 1.0, tau_user = 0.0, sigma_user = 0.0;
    void *pw_snap = nullptr, *pw_dh_base = nullptr;
    double *pw_part = nullptr;
    bool pw_base_valid = false;            // pw_dh_base holds the current base D-hat
    int64_t pw_last_k = -1;                // iterate index of the last update tried
    double pw_best_kkt = INFINITY;         // lowest KKT seen at an update point (FP32 iterates)
    int32_t dhat_mode = -1;                // mode D-hat was last formed with
    bool scaled = false;                   // aapdhg_set_scaling applied
    std::vector<double> dr_host, dc_host;  // Dr, Dc in internal order (when scaled)
    // raw device pointers kept for re-initialisation
    void *d_UP = nullptr;
    void *d_lo = nullptr;
    void *d_hi = nullptr;
    // chunk counters to zero at create
};

namespace {

aapdhg_status fail(aapdhg_t h, aapdhg_status s, const std::string &msg) {
    if (h) {
        if (h->sticky == AAPDHG_OK) {
            h->sticky = s;
            h->err = msg;
        }
    } else {
        g_create_err = msg;
    }
    return s;
}

#define CK(h, call)                                                                         \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail((h), AAPDHG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void *dev_alloc(aapdhg_t h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void *p = raw_alloc(bytes);
    if (p) {
        h->allocs.push_back({p, bytes});
        h->bytes += (int64_t)bytes;
    }
    return p;
}

void dev_free_all(aapdhg_t h) {
    for (auto &a : h->allocs) raw_free(a.p);
    h->allocs.clear();
    h->bytes = 0;
}

template <typename T>
T *alloc_copy(aapdhg_t h, const T *src, size_t count, bool *ok) {
    T *d = (T *)dev_alloc(h, sizeof(T) * count);
    if (!d) { *ok = false; return nullptr; }
    if (count && src &&
        cudaMemcpyAsync(d, src, sizeof(T) * count, cudaMemcpyHostToDevice, h->stream) != cudaSuccess) {
        *ok = false;
    }
    return d;
}

// ||v||_2^2 of a vector into st->scratch[slot] (last-block finalize).
template <typename V>
__global__ void __launch_bounds__(BLOCK) k_norm2(const V *v, int64_t len, double *part,
                                                 DevState *st, int slot) {
    __shared__ double sh[BLOCK];
    Acc<V> a;
    for (int64_t e = blockIdx.x * (int64_t)BLOCK + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * BLOCK)
        a.add_sq(v[e]);
    Acc<V> a1[1] = {a};
    block_reduce_store<V, 1>(a1, sh, part + blockIdx.x);
    if (last_block(&st->cnt_norm)) {
        const double s = block_sum_partials(part, gridDim.x, 1, 0, sh);
        if (threadIdx.x == 0) st->scratch[slot] = s;
    }
}

template <class K> int occupancy(K kernel) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, BLOCK, 0) != cudaSuccess) {
        cudaGetLastError();
        occ = 1;
    }
    return std::max(occ, 1);
}

template <typename V> Prob<V> &prob(aapdhg_t h);
template <> Prob<float> &prob<float>(aapdhg_t h) { return h->pf; }
template <> Prob<double> &prob<double>(aapdhg_t h) { return h->pd; }

int grid_for(aapdhg_t h, int64_t blocks_needed, int occ) {
    const int64_t cap = (int64_t)h->sm_count * std::max(occ, 1);
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks_needed, cap));
}

// D-hat (mode 1: the Remark on its construction; 0: identity) of the current K.
template <typename V> void launch_dhat(aapdhg_t h, int mode, cudaStream_t s) {
    Prob<V> &P = prob<V>(h);
    V *dh = const_cast<V *>(P.dh);
    const int64_t tasks = (int64_t)P.KT.n_chunks + P.KT.n_slices + P.K.n_chunks + P.K.n_slices;
    if (mode == 1) {          // the long rows' maxima start at 0
        if (P.KT.n_long) cudaMemsetAsync(dh, 0, sizeof(V) * P.KT.n_long, s);
        if (P.K.n_long) cudaMemsetAsync(dh + h->n, 0, sizeof(V) * P.K.n_long, s);
    }
    k_dhat_sliced<V><<<grid_for(h, (std::max(tasks, h->N / 32) + WARPS - 1) / WARPS, 8), BLOCK, 0, s>>>(
        P.KT, P.K, h->n, mode, dh);
    if (mode == 1 && P.KT.n_long + P.K.n_long > 0)
        k_dhat_long<V><<<grid_for(h, (P.KT.n_long + P.K.n_long + BLOCK - 1) / BLOCK, 4), BLOCK, 0, s>>>(
            P.KT.n_long, P.K.n_long, h->n, dh);
}

// Kernel kinds of the instrumentation.
enum { KIND_XSTEP = 0, KIND_YSTEP = 1, KIND_MEMORY = 2, KIND_MIX = 3, KIND_GRAM = 4, NKIND = 5 };

const char *const kKindName[NKIND] = {"aapdhg x-step", "aapdhg y-step", "aapdhg memory pass", "aapdhg AA mix",
                                      "aapdhg Gram pass"};

void mark_begin(aapdhg_t h, int kind) {
    h->launches += 1;
    nvtxRangePushA(kKindName[kind]);
    if (!h->prof_on) return;
    const size_t need = 2 * (h->ev_kind.size() + 1);
    while (h->ev.size() < need) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { h->prof_on = false; return; }
        h->ev.push_back(e);
    }
    cudaEventRecord(h->ev[2 * h->ev_kind.size()], h->stream);
    h->ev_kind.push_back(kind);
}

void mark_end(aapdhg_t h) {
    nvtxRangePop();
    if (!h->prof_on || h->ev_kind.empty()) return;
    cudaEventRecord(h->ev[2 * h->ev_kind.size() - 1], h->stream);
}

// Fold the recorded event pairs into the totals (after a stream sync).
void collect_marks(aapdhg_t h) {
    for (size_t i = 0; i < h->ev_kind.size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]) == cudaSuccess) {
            h->prof_ms[h->ev_kind[i]] += ms;
            h->prof_n[h->ev_kind[i]] += 1;
        }
    }
    h->ev_kind.clear();
}

// Fixed grids of the half-steps per task shape (deterministic reductions),
// sized for the common (non-KKT) variants, all of whose blocks are resident;
// a KKT launch (one in kkt_every) may run a short second wave.
template <typename V> void half_step_grids(aapdhg_t h) {
    Prob<V> &P = prob<V>(h);
    const int occx[NSHAPE] = {occupancy(k_xstep<V, false, 0>), occupancy(k_xstep<V, false, 1>),
                              occupancy(k_xstep<V, false, 2>), occupancy(k_xstep<V, false, 3>),
                              occupancy(k_xstep<V, false, 4>)};
    const int occy[NSHAPE] = {occupancy(k_ystep<V, false, 0>), occupancy(k_ystep<V, false, 1>),
                              occupancy(k_ystep<V, false, 2>), occupancy(k_ystep<V, false, 3>),
                              occupancy(k_ystep<V, false, 4>)};
    for (int sh = 0; sh < NSHAPE; ++sh) {
        const int g = task_shape(sh).g;
        h->gridx[sh] = grid_for(h, (P.KT.ntasks(g) + WARPS - 1) / WARPS, occx[sh]);
        h->gridy[sh] = grid_for(h, (P.K.ntasks(g) + WARPS - 1) / WARPS, occy[sh]);
    }
}

template <typename V>
aapdhg_status setup_device(aapdhg_t h, const HostCSR &K, const HostCSR &KT, const int8_t *sense,
                           const double *q, const double *c, const double *lb, const double *ub) {
    typedef typename Vec2<V>::T V2;
    Prob<V> &P = prob<V>(h);
    const int32_t m = h->m, n = h->n;
    const int64_t N = h->N, Z = h->nnz;
    bool ok = true;
    P.m = m;
    P.n = n;
    P.N = N;
    P.Npad = h->Npad;

    auto mk_csr = [&](const HostCSR &A, CSRView<V> &view, int which) {
        LayoutHost L;
        if (!build_layout(A, {RowSeg{0, A.rows, 0}}, L, h->lay[which])) { ok = false; return; }
        if (!upload_matrix<V>(A, view, [&](size_t b) { return dev_alloc(h, b); }, h->stream)) ok = false;
        std::vector<void *> &rec = h->lay_ptrs[which];
        auto track = [&](size_t b) {
            void *p = dev_alloc(h, b);
            if (p) rec.push_back(p);
            return p;
        };
        if (!upload_layout<V>(L, view, track, h->stream)) ok = false;
    };
    mk_csr(KT, P.KT, 0);
    mk_csr(K, P.K, 1);
    (void)Z;

    // vectors in internal order
    std::vector<V> cv(n), lov(N), hiv(N), qv(std::max(m, 1));
    for (int32_t j = 0; j < n; ++j) {
        const int32_t oj = h->perm_x[j];
        cv[j] = (V)c[oj];
        lov[j] = (V)lb[oj];
        hiv[j] = (V)ub[oj];
    }
    for (int32_t i = 0; i < m; ++i) {
        const int32_t oi = h->perm_y[i];
        qv[i] = (V)q[oi];
        lov[n + i] = sense[oi] == AAPDHG_ROW_GE ? V(0) : (V)(-INFINITY);
        hiv[n + i] = (V)INFINITY;
    }
    P.c = alloc_copy(h, cv.data(), cv.size(), &ok);
    P.q = alloc_copy(h, qv.data(), qv.size(), &ok);
    P.lo = alloc_copy(h, lov.data(), lov.size(), &ok);
    P.hi = alloc_copy(h, hiv.data(), hiv.size(), &ok);
    P.UP = (V2 *)dev_alloc(h, sizeof(V2) * N);
    P.dh = (V *)dev_alloc(h, sizeof(V) * N);
    P.g = (V *)dev_alloc(h, sizeof(V) * N);
    if (!P.UP || !P.dh || !P.g) ok = false;
    h->d_UP = P.UP;

    int occ3 = 0;
    half_step_grids<V>(h);
    // partial-sum buffers for any grid of resident blocks (a later layout may
    // need more blocks than this one)
    const int gmax1 = h->sm_count * 8, gmax2 = h->sm_count * 8;
    P.grid1 = h->gridx[0];
    P.grid2 = h->gridy[0];
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ3, k_memory<V>, BLOCK, 0);

    P.grid3 = grid_for(h, (N + BLOCK - 1) / BLOCK, std::max(occ3, 1));
    h->grid5 = grid_for(h, (N + BLOCK - 1) / BLOCK, 4);
    P.part1 = (double *)dev_alloc(h, sizeof(double) * 4 * gmax1);
    P.part2 = (double *)dev_alloc(h, sizeof(double) * 3 * gmax2);
    P.part3 = (double *)dev_alloc(h, sizeof(double) * (MAXM + 3) * h->sm_count * 8);
    P.part4 = (double *)dev_alloc(h, sizeof(double) * GRAM_MAXPAIRS * h->sm_count * GRAM_MAX_OCC);
    h->st = (DevState *)dev_alloc(h, sizeof(DevState));
    P.st = h->st;
    if (!P.part1 || !P.part2 || !P.part3 || !P.part4 || !h->st) ok = false;
    if (!ok) return fail(h, AAPDHG_ERR_OOM, "device allocation or copy failed during create");
    CK(h, cudaMemsetAsync(h->st, 0, sizeof(DevState), h->stream));
    P.DG = P.W = nullptr;
    P.sc_x = P.sc_y = nullptr;
    P.tr = Trace{0, nullptr, nullptr, nullptr, nullptr};

    // D-hat and the norms ||q||, ||c|| on the device
    const int gE = grid_for(h, (N + BLOCK - 1) / BLOCK, 4);
    launch_dhat<V>(h, 1, h->stream);
    h->dhat_mode = 1;
    k_norm2<V><<<gE, BLOCK, 0, h->stream>>>(P.q, m, P.part3, h->st, 0);
    k_norm2<V><<<gE, BLOCK, 0, h->stream>>>(P.c, n, P.part3, h->st, 1);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(h->st_host, h->st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->mp.q_norm = sqrt(h->st_host->scratch[0]);
    h->mp.c_norm = sqrt(h->st_host->scratch[1]);
    return AAPDHG_OK;
}

// (Re)size the Anderson rings for memory M.
template <typename V> aapdhg_status ensure_rings(aapdhg_t h, int32_t M) {
    Prob<V> &P = prob<V>(h);
    if (M == 0 || (P.DG && h->ring_mem >= M)) return AAPDHG_OK;
    // rings always hold NSLOT slots: allocate once at full size
    P.DG = (V *)dev_alloc(h, sizeof(V) * (size_t)NSLOT * h->Npad);
    P.W = (V *)dev_alloc(h, sizeof(V) * (size_t)NSLOT * h->Npad);
    if (!P.DG || !P.W) return fail(h, AAPDHG_ERR_OOM, "device allocation of the Anderson memory failed");
    h->ring_mem = MAXM;
    return AAPDHG_OK;
}

void drop_graphs(aapdhg_t h);

template <typename V> aapdhg_status reset_run(aapdhg_t h) {
    h->time_used = 0.0;
    typedef typename Vec2<V>::T V2;
    Prob<V> &P = prob<V>(h);
    const int32_t n = h->n, m = h->m;
    std::vector<V2> up(h->N);
    for (int32_t j = 0; j < n; ++j) {
        const int32_t oj = h->perm_x[j];
        up[j].x = (V)(h->scaled ? h->x0[oj] / h->dc_host[j] : h->x0[oj]);
        up[j].y = V(0);
    }
    for (int32_t i = 0; i < m; ++i) {
        const int32_t oi = h->perm_y[i];
        up[n + i].x = (V)(h->scaled ? h->y0[oi] / h->dr_host[i] : h->y0[oi]);
        up[n + i].y = V(0);
    }
    CK(h, cudaMemcpyAsync(P.UP, up.data(), sizeof(V2) * h->N, cudaMemcpyHostToDevice, h->stream));
    // clear the run fields of the state, keep the norm scratch
    CK(h, cudaMemsetAsync(h->st, 0, offsetof(DevState, scratch), h->stream));
    if (h->pw_period > 0) {
        // a run starts with the given steps and the base D-hat (R13)
        h->mp.tau = h->tau_user;
        h->mp.sigma = h->sigma_user;
        h->pw_gamma = sqrt(h->tau_user * h->sigma_user);
        h->pw_omega = h->tau_user > 0 ? sqrt(h->sigma_user / h->tau_user) : 1.0;
        h->pw_last_k = -1;
        h->pw_best_kkt = INFINITY;
        if (h->pw_dh_base) {
            V *dh = const_cast<V *>(P.dh);
            if (!h->pw_base_valid) {
                CK(h, cudaMemcpyAsync(h->pw_dh_base, dh, sizeof(V) * h->N, cudaMemcpyDeviceToDevice, h->stream));
                h->pw_base_valid = true;
            } else {
                CK(h, cudaMemcpyAsync(dh, h->pw_dh_base, sizeof(V) * h->N, cudaMemcpyDeviceToDevice, h->stream));
            }
        }
        drop_graphs(h);
    }
    if (P.tr.cap > 0) {
        std::vector<int8_t> b(P.tr.cap, -1);
        std::vector<double> nanv(P.tr.cap, NAN);
        std::vector<int32_t> mk(P.tr.cap, -1);
        CK(h, cudaMemcpyAsync(P.tr.branch, b.data(), P.tr.cap, cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaMemcpyAsync(P.tr.gnorm, nanv.data(), 8 * P.tr.cap, cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaMemcpyAsync(P.tr.kkt, nanv.data(), 8 * P.tr.cap, cudaMemcpyHostToDevice, h->stream));
        CK(h, cudaMemcpyAsync(P.tr.mk, mk.data(), 4 * P.tr.cap, cudaMemcpyHostToDevice, h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return AAPDHG_OK;
}

// The device stopped the run: st->error 1 = NaN/Inf met, 2 = a bounded wait
// of the Gram pass on its bulk copies gave up.
aapdhg_status device_error(aapdhg_t h) {
    if (h->st_host->error == 2)
        return fail(h, AAPDHG_ERR_CUDA, "a bounded device-side wait (Gram pass copies) gave up");
    return fail(h, AAPDHG_ERR_NUMERIC, "NaN or Inf in the iterate");
}

aapdhg_status reset_any(aapdhg_t h) {
    return h->prec == AAPDHG_FP64 ? reset_run<double>(h) : reset_run<float>(h);
}

template <typename V, int MC> void launch_memory_mix(aapdhg_t h, int mode, int fin) {
    Prob<V> &P = prob<V>(h);
    const int M = (h->mp.method == 0) ? 0 : h->mp.mem;
    // grids of the memory and Gram passes for this instance: all resident
    // blocks (fixed per instance, so their block partials are summed in a
    // fixed order)
    static int occ_mem = 0, occ_mix = 0, occ_gram = 0;
    if (occ_mem == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_mem, k_memory<V>, BLOCK, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_mix, k_mix<V, MC>, BLOCK, 0);
        cudaFuncSetAttribute(k_gram<V>, cudaFuncAttributeMaxDynamicSharedMemorySize, gram_dyn_smem(MAXM));
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_gram, k_gram<V>, BLOCK, gram_dyn_smem(MC));
        occ_mem = std::max(occ_mem, 1);
        occ_mix = std::max(occ_mix, 1);
        occ_gram = std::min(std::max(occ_gram, 1), GRAM_MAX_OCC);
    }
    P.grid3 = M > 0 ? grid_for(h, (h->N + BLOCK * 4 - 1) / (BLOCK * 4), occ_mem) : 1;
    P.grid4 = M > 0 ? grid_for(h, (h->N + 127) / 128, occ_gram) : 1;
    const int g5 = grid_for(h, (h->N + BLOCK * 4 - 1) / (BLOCK * 4), occ_mix);
    const int g3 = P.grid3;
    mark_begin(h, KIND_MEMORY);
    // fin with a memory: one more block runs the half-steps' final reduction
    // beside the streaming blocks
    k_memory<V><<<g3 + ((fin && M > 0) ? 1 : 0), BLOCK, 0, h->stream>>>(P, h->mp, mode, fin);
    mark_end(h);
    if (mode == MODE_ITER && M > 0) {
        mark_begin(h, KIND_GRAM);
        k_gram<V><<<P.grid4, BLOCK, gram_dyn_smem(M), h->stream>>>(P, h->mp);
        mark_end(h);
        mark_begin(h, KIND_MIX);
        k_mix<V, MC><<<g5, BLOCK, 0, h->stream>>>(P, h->mp);
        mark_end(h);
    }
}

template <typename V, bool KKT> void launch_x(aapdhg_t h, int shape, int mode) {
    Prob<V> &P = prob<V>(h);
    if (shape == 1) k_xstep<V, KKT, 1><<<P.grid1, BLOCK, 0, h->stream>>>(P, h->mp, mode);
    else if (shape == 2) k_xstep<V, KKT, 2><<<P.grid1, BLOCK, 0, h->stream>>>(P, h->mp, mode);
    else if (shape == 3) k_xstep<V, KKT, 3><<<P.grid1, BLOCK, 0, h->stream>>>(P, h->mp, mode);
    else if (shape == 4) k_xstep<V, KKT, 4><<<P.grid1, BLOCK, 0, h->stream>>>(P, h->mp, mode);
    else k_xstep<V, KKT, 0><<<P.grid1, BLOCK, 0, h->stream>>>(P, h->mp, mode);
}

template <typename V, bool KKT> void launch_y(aapdhg_t h, int shape, int mode) {
    Prob<V> &P = prob<V>(h);
    if (shape == 1) k_ystep<V, KKT, 1><<<P.grid2, BLOCK, 0, h->stream>>>(P, h->mp, mode);
    else if (shape == 2) k_ystep<V, KKT, 2><<<P.grid2, BLOCK, 0, h->stream>>>(P, h->mp, mode);
    else if (shape == 3) k_ystep<V, KKT, 3><<<P.grid2, BLOCK, 0, h->stream>>>(P, h->mp, mode);
    else if (shape == 4) k_ystep<V, KKT, 4><<<P.grid2, BLOCK, 0, h->stream>>>(P, h->mp, mode);
    else k_ystep<V, KKT, 0><<<P.grid2, BLOCK, 0, h->stream>>>(P, h->mp, mode);
}

template <typename V> void launch_T(aapdhg_t h, bool kkt, int mode, bool with_finalize = true) {
    mark_begin(h, KIND_XSTEP);
    if (kkt) launch_x<V, true>(h, h->shape_x, mode);
    else launch_x<V, false>(h, h->shape_x, mode);
    mark_end(h);
    mark_begin(h, KIND_YSTEP);                 // the y-step and its final reduction
    if (kkt) launch_y<V, true>(h, h->shape_y, mode);
    else launch_y<V, false>(h, h->shape_y, mode);
    if (with_finalize) {
        k_finalize<V><<<1, BLOCK, 0, h->stream>>>(prob<V>(h), h->mp, mode, kkt ? 1 : 0);
        h->launches += 1;
    }
    mark_end(h);
}

void set_shapes(aapdhg_t h, int sx, int sy) {
    h->shape_x = sx;
    h->shape_y = sy;
    h->pf.grid1 = h->pd.grid1 = h->gridx[sx];
    h->pf.grid2 = h->pd.grid2 = h->gridy[sy];
}

void drop_graphs(aapdhg_t h);

// Autotuning of the two half-step kernels: every compiled task shape is
// launched on the handle's matrices (timing mode: T(u) goes to the scratch
// component, no run state changes), twice to warm up and five times under
// CUDA events; the fastest shape of each kernel is kept.
template <typename V> aapdhg_status autotune_t(aapdhg_t h) {
    Prob<V> &P = prob<V>(h);
    cudaEvent_t e0, e1;
    CK(h, cudaEventCreate(&e0));
    CK(h, cudaEventCreate(&e1));
    // two interleaved rounds, the faster of the two kept per shape (robust to
    // clock ramps and to whatever ran just before)
    double tx[NSHAPE], ty[NSHAPE];
    for (int sh = 0; sh < NSHAPE; ++sh) tx[sh] = ty[sh] = 1e30;
    for (int round = 0; round < 2; ++round)
        for (int sh = 0; sh < NSHAPE; ++sh) {
            P.grid1 = h->gridx[sh];
            P.grid2 = h->gridy[sh];
            float ms = 0.f;
            for (int w = 0; w < 2; ++w) launch_x<V, false>(h, sh, MODE_TUNE);
            cudaEventRecord(e0, h->stream);
            for (int r = 0; r < 5; ++r) launch_x<V, false>(h, sh, MODE_TUNE);
            cudaEventRecord(e1, h->stream);
            CK(h, cudaEventSynchronize(e1));
            cudaEventElapsedTime(&ms, e0, e1);
            tx[sh] = std::min(tx[sh], 1e3 * ms / 5);
            for (int w = 0; w < 2; ++w) launch_y<V, false>(h, sh, MODE_TUNE);
            cudaEventRecord(e0, h->stream);
            for (int r = 0; r < 5; ++r) launch_y<V, false>(h, sh, MODE_TUNE);
            cudaEventRecord(e1, h->stream);
            CK(h, cudaEventSynchronize(e1));
            cudaEventElapsedTime(&ms, e0, e1);
            ty[sh] = std::min(ty[sh], 1e3 * ms / 5);
        }
    int bx = 0, by = 0;
    for (int sh = 0; sh < NSHAPE; ++sh) {
        h->tune_us[sh] = tx[sh];
        h->tune_us[NSHAPE + sh] = ty[sh];
        if (tx[sh] < tx[bx]) bx = sh;
        if (ty[sh] < ty[by]) by = sh;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(h, cudaGetLastError());
    set_shapes(h, bx, by);
    h->tuned = true;
    drop_graphs(h);
    return AAPDHG_OK;
}

// ---------------------------------------------------------------------------
// Layout of K' and K: the slice width limit (rows up to it go to SELL-32
// slices, one lane per row) and the entries per warp task of a longer row.
// ---------------------------------------------------------------------------
void dev_free_ptrs(aapdhg_t h, const std::vector<void *> &ptrs) {
    for (void *p : ptrs)
        for (size_t i = 0; i < h->allocs.size(); ++i)
            if (h->allocs[i].p == p) {
                h->bytes -= (int64_t)h->allocs[i].bytes;
                raw_free(p);
                h->allocs.erase(h->allocs.begin() + (long)i);
                break;
            }
}

// The internal CSR of a matrix as the device holds it (in the iterate
// precision; scaled when the LP was scaled).
template <typename V> aapdhg_status download_csr(aapdhg_t h, const CSRView<V> &v, int64_t nnz, HostCSR &A) {
    A.rows = v.rows;
    A.rp.resize((size_t)v.rows + 1);
    A.ci.resize((size_t)nnz);
    A.val.resize((size_t)nnz);
    std::vector<V> tmp((size_t)std::max<int64_t>(nnz, 1));
    CK(h, cudaMemcpyAsync(A.rp.data(), v.rp, sizeof(int32_t) * ((size_t)v.rows + 1), cudaMemcpyDeviceToHost,
                          h->stream));
    if (nnz > 0) {
        CK(h, cudaMemcpyAsync(A.ci.data(), v.ci, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaMemcpyAsync(tmp.data(), v.val, sizeof(V) * (size_t)nnz, cudaMemcpyDeviceToHost, h->stream));
    }
    CK(h, cudaStreamSynchronize(h->stream));
    for (int64_t k = 0; k < nnz; ++k) A.val[k] = (double)tmp[k];
    return AAPDHG_OK;
}

// Rebuild the layouts of K' (prm[0]) and K (prm[1]); the run state is kept,
// the task shapes are tuned again at the next iterate.
template <typename V> aapdhg_status set_layout_t(aapdhg_t h, const LayoutParams (&prm)[2]) {
    Prob<V> &P = prob<V>(h);
    CK(h, cudaStreamSynchronize(h->stream));
    HostCSR A[2];
    aapdhg_status s = download_csr<V>(h, P.KT, h->nnz, A[0]);
    if (s == AAPDHG_OK) s = download_csr<V>(h, P.K, h->nnz, A[1]);
    if (s != AAPDHG_OK) return s;
    CSRView<V> nv[2] = {P.KT, P.K};
    std::vector<void *> rec[2];
    bool ok = true;
    for (int w = 0; w < 2 && ok; ++w) {
        LayoutHost L;
        if (!build_layout(A[w], {RowSeg{0, A[w].rows, 0}}, L, prm[w])) { ok = false; break; }
        auto track = [&](size_t b) {
            void *p = dev_alloc(h, b);
            if (p) rec[w].push_back(p);
            return p;
        };
        if (!upload_layout<V>(L, nv[w], track, h->stream)) ok = false;
    }
    if (!ok) {
        dev_free_ptrs(h, rec[0]);
        dev_free_ptrs(h, rec[1]);
        return fail(h, AAPDHG_ERR_OOM, "layout: device allocation or copy failed");
    }
    dev_free_ptrs(h, h->lay_ptrs[0]);
    dev_free_ptrs(h, h->lay_ptrs[1]);
    h->lay_ptrs[0] = rec[0];
    h->lay_ptrs[1] = rec[1];
    P.KT = nv[0];
    P.K = nv[1];
    h->lay[0] = prm[0];
    h->lay[1] = prm[1];
    half_step_grids<V>(h);
    set_shapes(h, 0, 0);
    h->tuned = false;
    drop_graphs(h);
    return AAPDHG_OK;
}

static_assert(kNumLayoutCand == AAPDHG_LAYOUT_CANDIDATES, "layout candidates of the C ABI and the tuner differ");

// Every candidate layout (the same for both matrices), with the task shapes
// tuned on it.  The x-step reads only K' and the y-step only K, so K' keeps
// the candidate with the fastest x-step and K the one with the fastest
// y-step.
template <typename V> aapdhg_status autotune_layout_t(aapdhg_t h) {
    double bestx = INFINITY, besty = INFINITY;
    int bx_i = 0, by_i = 0;
    for (int c = 0; c < AAPDHG_LAYOUT_CANDIDATES; ++c) {
        const LayoutParams both[2] = {kLayoutCand[c], kLayoutCand[c]};
        aapdhg_status s = set_layout_t<V>(h, both);
        if (s == AAPDHG_OK) s = autotune_t<V>(h);
        if (s != AAPDHG_OK) return s;
        double bx = INFINITY, by = INFINITY;
        for (int sh = 0; sh < NSHAPE; ++sh) {
            bx = std::min(bx, h->tune_us[sh]);
            by = std::min(by, h->tune_us[NSHAPE + sh]);
        }
        h->lay_us[2 * c] = bx;
        h->lay_us[2 * c + 1] = by;
        if (bx < bestx) { bestx = bx; bx_i = c; }
        if (by < besty) { besty = by; by_i = c; }
    }
    const LayoutParams chosen[2] = {kLayoutCand[bx_i], kLayoutCand[by_i]};
    aapdhg_status s = set_layout_t<V>(h, chosen);
    if (s == AAPDHG_OK) s = autotune_t<V>(h);
    return s;
}

template <typename V> void launch_memory_any(aapdhg_t h, int mode, int fin) {
    const int M = h->mp.mem;
    if (M <= 4) launch_memory_mix<V, 4>(h, mode, fin);
    else if (M <= 8) launch_memory_mix<V, 8>(h, mode, fin);
    else if (M <= 16) launch_memory_mix<V, 16>(h, mode, fin);
    else if (M <= 20) launch_memory_mix<V, 20>(h, mode, fin);
    else launch_memory_mix<V, 32>(h, mode, fin);
}

// One loop iteration.  Without a KKT test (the iteration cannot stop) the
// half-steps' final reduction runs in the memory pass's last block instead
// of a launch of its own.
template <typename V> void launch_iteration(aapdhg_t h, bool kkt, int mode) {
    const bool fuse = mode == MODE_ITER && !kkt;
    launch_T<V>(h, kkt, mode, !fuse);
    if (mode != MODE_EVAL) launch_memory_any<V>(h, mode, fuse ? 1 : 0);
}

aapdhg_status read_state(aapdhg_t h, bool full = true) {
    const size_t bytes = full ? sizeof(DevState) : offsetof(DevState, list);
    CK(h, cudaMemcpyAsync(h->st_host, h->st, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    collect_marks(h);
    return AAPDHG_OK;
}

void drop_graphs(aapdhg_t h) {
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
}

// Launch one full chunk of CHUNK_ITERS iterations starting at iteration `hit`
// as a CUDA graph (captured once per KKT phase on a private stream, replayed
// on the handle's stream).  Returns false when graphs are not usable.
template <typename V> bool launch_chunk_graph(aapdhg_t h, int64_t hit, int32_t kkt_every) {
    if (!h->use_graphs || h->prof_on) return false;
    const int64_t phase = kkt_every > 0 ? hit % kkt_every : 0;
    const double tol = h->mp.tol;
    for (auto &g : h->graphs)
        if (g.phase == phase && g.kkt_every == kkt_every && g.tol == tol) {
            if (cudaGraphLaunch(g.exec, h->stream) != cudaSuccess) { cudaGetLastError(); return false; }
            h->launches += g.kernels;
            return true;
        }
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        h->use_graphs = false;
        return false;
    }
    if (h->graphs.size() >= 8) drop_graphs(h);
    cudaStream_t user = h->stream;
    h->stream = h->cap_stream;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    const int64_t saved = h->launches;
    if (ok) {
        for (int64_t c = 0; c < CHUNK_ITERS; ++c) {
            const bool kkt = kkt_every > 0 && ((hit + c) % kkt_every) == 0;
            launch_iteration<V>(h, kkt, MODE_ITER);
        }
        ok = cudaStreamEndCapture(h->cap_stream, &graph) == cudaSuccess;
    }
    h->stream = user;
    const int64_t kernels = h->launches - saved;
    h->launches = saved;
    cudaGraphExec_t exec = nullptr;
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        h->use_graphs = false;
        return false;
    }
    h->graphs.push_back({exec, phase, kkt_every, tol, kernels});
    if (cudaGraphLaunch(exec, h->stream) != cudaSuccess) { cudaGetLastError(); return false; }
    h->launches += kernels;
    return true;
}

// Primal weight update at the iterate u^k (Alg. "Primal weight update",
// readings R13-R15): Delta_x, Delta_y against the snapshot (which becomes
// u^k); when both exceed epsilon_zero, the new omega gives tau = gamma/omega,
// sigma = gamma omega, D-hat is re-blended (Remark on the form) and the memory
// restarts at this iteration.
template <typename V> aapdhg_status pw_update(aapdhg_t h, int64_t k) {
    Prob<V> &P = prob<V>(h);
    const int cur = (int)(((k - 1) & 1) ^ 1);
    k_pw_delta<V><<<h->grid5, BLOCK, 0, h->stream>>>(P.UP, (V *)h->pw_snap, h->n, h->N, cur, 0,
                                                      h->pw_part, h->st);
    CK(h, cudaGetLastError());
    aapdhg_status s = read_state(h);
    if (s != AAPDHG_OK) return s;
    const double dx = sqrt(h->st_host->scratch[2]), dy = sqrt(h->st_host->scratch[3]);
    // FP32 iterates: an update only while the run still improves, i.e. the
    // last KKT test is below every one seen at earlier update points.  At
    // FP32's attainable accuracy Delta_x, Delta_y are rounding noise, and an
    // omega driven by them drifts until sigma amplifies the FP32 error of
    // q - Kx into y (a run diverges).  The paper works in FP64; the FP64
    // path applies every update.
    bool improving = true;
    if (sizeof(V) == 4 && h->mp.kkt_every > 0 && h->st_host->kkt_valid) {
        const double kk = h->st_host->kkt[3];
        improving = kk < h->pw_best_kkt;
        h->pw_best_kkt = std::min(h->pw_best_kkt, kk);
    }
    if (!(dx > h->pw_eps && dy > h->pw_eps) || !improving) return AAPDHG_OK;
    h->pw_omega = exp(h->pw_theta * log(dy / dx) + (1.0 - h->pw_theta) * log(h->pw_omega));
    h->mp.tau = h->pw_gamma / h->pw_omega;
    h->mp.sigma = h->pw_gamma * h->pw_omega;
    if (h->pw_dhat && h->pw_dh_base) {
        const double r1 = h->st_host->gnorm, r2 = h->st_host->gnorm_prev;
        const double rho = std::isnan(r2) ? 0.0 : (r2 - r1) / std::max(r2, h->pw_eps);
        const double alpha = rho >= h->pw_rho_min ? h->pw_alpha_dec : h->pw_alpha_inc;
        k_dhat_blend<V><<<h->grid5, BLOCK, 0, h->stream>>>(const_cast<V *>(P.dh), (const V *)h->pw_dh_base,
                                                            h->n, h->N, h->pw_omega, alpha);
        CK(h, cudaGetLastError());
    }
    const int32_t one = 1;
    CK(h, cudaMemcpyAsync(&h->st->restart, &one, sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    drop_graphs(h);
    return AAPDHG_OK;
}

template <typename V> aapdhg_status iterate_t(aapdhg_t h, int64_t max_iters, double tol,
                                              int32_t kkt_every, int64_t *done_iters) {
    Prob<V> &P = prob<V>(h);
    h->mp.tol = tol;
    h->mp.kkt_every = kkt_every;
    aapdhg_status s = ensure_rings<V>(h, (h->mp.method == 0) ? 0 : h->mp.mem);
    if (s != AAPDHG_OK) return s;
    if (h->autotune && !h->tuned && (s = autotune_t<V>(h)) != AAPDHG_OK) return s;
    if ((s = read_state(h)) != AAPDHG_OK) return s;
    if (!h->st_host->init_done) {
        if (h->pw_period > 0)      // snapshot u^0 for the first primal weight update
            k_pw_delta<V><<<h->grid5, BLOCK, 0, h->stream>>>(P.UP, (V *)h->pw_snap, h->n, h->N, 0, 1,
                                                              h->pw_part, h->st);
        launch_iteration<V>(h, false, MODE_INIT);
        CK(h, cudaGetLastError());
        if ((s = read_state(h)) != AAPDHG_OK) return s;
    }
    if (h->st_host->error) return device_error(h);
    // a new call re-tests the current iterate against its own tolerance
    CK(h, cudaMemsetAsync(&h->st->done, 0, sizeof(int32_t), h->stream));
    const int64_t it0 = h->st_host->it;
    int64_t hit = it0, launched = 0;
    bool done = false;
    const auto t_start = std::chrono::steady_clock::now();
    while (launched < max_iters && !done) {
        if (h->time_limit > 0.0) {
            // checked between chunks, after the last chunk's state was read
            const double t = h->time_used +
                std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
            if (t > h->time_limit) {
                h->time_used = t;
                if (done_iters) *done_iters = hit - it0;
                return AAPDHG_ERR_TIMEOUT;
            }
        }
        int64_t chunk = std::min<int64_t>(CHUNK_ITERS, max_iters - launched);
        if (h->pw_period > 0) {
            // the current iterate is u^k with k = hit + 1; updates at k = 0 mod U_P,
            // each at the start of a chunk
            const int64_t k = hit + 1, r = k % h->pw_period;
            if (r == 0 && h->pw_last_k != k) {
                if ((s = pw_update<V>(h, k)) != AAPDHG_OK) return s;
                h->pw_last_k = k;
            }
            chunk = std::min<int64_t>(chunk, r == 0 ? h->pw_period : h->pw_period - r);
        }
        if (!(chunk == CHUNK_ITERS && launch_chunk_graph<V>(h, hit, kkt_every))) {
            for (int64_t c = 0; c < chunk; ++c) {
                const int64_t itc = hit + c;
                const bool kkt = kkt_every > 0 && (itc % kkt_every) == 0;
                launch_iteration<V>(h, kkt, MODE_ITER);
            }
        }
        CK(h, cudaGetLastError());
        launched += chunk;
        if ((s = read_state(h, false)) != AAPDHG_OK) return s;
        if (h->st_host->error) return device_error(h);
        done = h->st_host->done != 0;
        hit = h->st_host->it;
    }
    (void)P;
    h->time_used += std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    if (done_iters) *done_iters = hit - it0;
    if (done) return AAPDHG_OK;
    // max_iters may also end exactly on a converged iterate that was not tested
    return AAPDHG_NOT_CONVERGED;
}

template <typename V> aapdhg_status get_iterate_t(aapdhg_t h, double *x, double *y) {
    typedef typename Vec2<V>::T V2;
    Prob<V> &P = prob<V>(h);
    aapdhg_status s = read_state(h);
    if (s != AAPDHG_OK) return s;
    const int cur = h->st_host->init_done ? (int)((h->st_host->it & 1) ^ 1) : 0;
    std::vector<V2> up(h->N);
    CK(h, cudaMemcpyAsync(up.data(), P.UP, sizeof(V2) * h->N, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (x)
        for (int32_t j = 0; j < h->n; ++j) {
            const double v = (double)(cur ? up[j].y : up[j].x);
            x[h->perm_x[j]] = h->scaled ? v * h->dc_host[j] : v;      // x = Dc x~
        }
    if (y)
        for (int32_t i = 0; i < h->m; ++i) {
            const double v = (double)(cur ? up[h->n + i].y : up[h->n + i].x);
            y[h->perm_y[i]] = h->scaled ? v * h->dr_host[i] : v;      // y = Dr y~
        }
    return AAPDHG_OK;
}

// The Anderson memory as the device holds it after the last iteration: the
// Gram matrix and right-hand side in list order, the dG columns and g^k in
// the caller's element order (FP32 values widened exactly in mixed mode).
template <typename V> aapdhg_status get_memory_t(aapdhg_t h, int32_t capacity, int32_t *count,
                                                 double *gram, double *rhs, double *dg, double *g) {
    Prob<V> &P = prob<V>(h);
    aapdhg_status s = read_state(h);
    if (s != AAPDHG_OK) return s;
    const DevState &st = *h->st_host;
    const int k = (h->mp.method == 0 || h->mp.mem == 0 || !P.DG || !st.init_done) ? 0 : st.count;
    if (count) *count = k;
    if (k > capacity) return fail(h, AAPDHG_ERR_INVALID, "get_memory: capacity below the column count");
    const int32_t n = h->n, m = h->m;
    const int64_t N = h->N;
    for (int a = 0; a < k; ++a) {
        if (rhs) rhs[a] = st.rhs[st.list[a]];
        if (gram)
            for (int b = 0; b < k; ++b) gram[a * k + b] = st.G[st.list[a] * NSLOT + st.list[b]];
    }
    std::vector<V> col(N);
    auto to_caller = [&](double *out) {
        for (int32_t j = 0; j < n; ++j) out[h->perm_x[j]] = (double)col[j];
        for (int32_t i = 0; i < m; ++i) out[n + h->perm_y[i]] = (double)col[n + i];
    };
    if (dg)
        for (int a = 0; a < k; ++a) {
            CK(h, cudaMemcpyAsync(col.data(), P.DG + (int64_t)st.list[a] * P.Npad, sizeof(V) * N,
                                  cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
            to_caller(dg + (int64_t)a * N);
        }
    if (g) {
        CK(h, cudaMemcpyAsync(col.data(), P.g, sizeof(V) * N, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        to_caller(g);
    }
    return AAPDHG_OK;
}

template <typename V> aapdhg_status get_kkt_t(aapdhg_t h, double *out6) {
    launch_iteration<V>(h, true, MODE_EVAL);
    CK(h, cudaGetLastError());
    aapdhg_status s = read_state(h);
    if (s != AAPDHG_OK) return s;
    for (int k = 0; k < 6; ++k) out6[k] = h->st_host->kkt[k];
    return AAPDHG_OK;
}

template <typename V> aapdhg_status estimate_norm_t(aapdhg_t h, int32_t iters, uint64_t seed,
                                                   double *norm) {
    Prob<V> &P = prob<V>(h);
    const int32_t n = h->n, m = h->m;
    V *v = (V *)dev_alloc(h, sizeof(V) * n);
    V *w = (V *)dev_alloc(h, sizeof(V) * std::max(m, 1));
    double *part = (double *)dev_alloc(h, sizeof(double) * std::max(P.grid1, P.grid2));
    if (!v || !w || !part) return fail(h, AAPDHG_ERR_OOM, "power iteration buffers");
    std::vector<V> hv(n);
    uint64_t z = seed ? seed : 0x9E3779B97F4A7C15ull;
    for (int32_t j = 0; j < n; ++j) {     // splitmix64 uniform in [-1, 1)
        z += 0x9E3779B97F4A7C15ull;
        uint64_t t = z;
        t = (t ^ (t >> 30)) * 0xBF58476D1CE4E5B9ull;
        t = (t ^ (t >> 27)) * 0x94D049BB133111EBull;
        t ^= t >> 31;
        hv[j] = (V)((double)(t >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
    }
    CK(h, cudaMemcpyAsync(v, hv.data(), sizeof(V) * n, cudaMemcpyHostToDevice, h->stream));
    std::vector<double> hp(std::max(P.grid1, P.grid2));
    double lam = 0.0;
    for (int32_t t = 0; t < iters; ++t) {
        if (m > 0) k_spmv_plain<V><<<P.grid2, BLOCK, 0, h->stream>>>(P.K, v, w, part);
        k_spmv_plain<V><<<P.grid1, BLOCK, 0, h->stream>>>(P.KT, w, v, part);
        CK(h, cudaGetLastError());
        CK(h, cudaMemcpyAsync(hp.data(), part, sizeof(double) * P.grid1, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
        double s = 0.0;
        for (int b = 0; b < P.grid1; ++b) s += hp[b];
        lam = sqrt(s);                   // ||K'K v|| for the unit v of this step
        k_scale<V><<<grid_for(h, (n + BLOCK - 1) / BLOCK, 4), BLOCK, 0, h->stream>>>(v, n, part, P.grid1);
        CK(h, cudaGetLastError());
    }
    CK(h, cudaStreamSynchronize(h->stream));
    // free the scratch (last three allocations)
    for (int k = 0; k < 3; ++k) {
        DevAlloc a = h->allocs.back();
        h->allocs.pop_back();
        h->bytes -= (int64_t)a.bytes;
        if (g_free) g_free(a.p, g_ctx); else cudaFree(a.p);
    }
    *norm = sqrt(lam);
    return AAPDHG_OK;
}

template <typename V> aapdhg_status set_scaling_t(aapdhg_t h, int32_t ruiz_iters, int32_t pc) {
    Prob<V> &P = prob<V>(h);
    const int32_t m = h->m, n = h->n;
    V *dr = (V *)dev_alloc(h, sizeof(V) * std::max(m, 1));
    V *dc = (V *)dev_alloc(h, sizeof(V) * n);
    V *tr = (V *)dev_alloc(h, sizeof(V) * std::max(m, 1));
    V *tc = (V *)dev_alloc(h, sizeof(V) * n);
    V *scx = (V *)dev_alloc(h, sizeof(V) * n);
    V *scy = (V *)dev_alloc(h, sizeof(V) * std::max(m, 1));
    if (!dr || !dc || !tr || !tc || !scx || !scy) return fail(h, AAPDHG_ERR_OOM, "scaling buffers");
    cudaStream_t s = h->stream;
    const int gv = grid_for(h, (h->N + BLOCK - 1) / BLOCK, 4);
    const int gr = grid_for(h, (h->N + WARPS - 1) / WARPS, 8);
    k_fill<V><<<gv, BLOCK, 0, s>>>(dr, V(1), m);
    k_fill<V><<<gv, BLOCK, 0, s>>>(dc, V(1), n);
    for (int32_t pass = 0; pass < ruiz_iters + (pc ? 1 : 0); ++pass) {
        const int sum = pass >= ruiz_iters;          // the last pass is Pock-Chambolle
        if (m > 0) k_row_norm<V><<<gr, BLOCK, 0, s>>>(P.K, sum, tr);
        k_row_norm<V><<<gr, BLOCK, 0, s>>>(P.KT, sum, tc);
        k_factor<V><<<gv, BLOCK, 0, s>>>(tr, m);
        k_factor<V><<<gv, BLOCK, 0, s>>>(tc, n);
        if (m > 0) k_scale_matrix<V><<<gr, BLOCK, 0, s>>>(P.K, tr, tc);
        k_scale_matrix<V><<<gr, BLOCK, 0, s>>>(P.KT, tc, tr);
        k_vmul<V><<<gv, BLOCK, 0, s>>>(dr, tr, m);
        k_vmul<V><<<gv, BLOCK, 0, s>>>(dc, tc, n);
    }
    k_vmul<V><<<gv, BLOCK, 0, s>>>(const_cast<V *>(P.c), dc, n);
    k_vmul<V><<<gv, BLOCK, 0, s>>>(const_cast<V *>(P.q), dr, m);
    k_vdiv<V><<<gv, BLOCK, 0, s>>>(const_cast<V *>(P.lo), dc, n);   // x part of the bounds
    k_vdiv<V><<<gv, BLOCK, 0, s>>>(const_cast<V *>(P.hi), dc, n);
    k_vinv<V><<<gv, BLOCK, 0, s>>>(scx, dc, n);
    k_vinv<V><<<gv, BLOCK, 0, s>>>(scy, dr, m);
    CK(h, cudaGetLastError());
    std::vector<V> hr(std::max(m, 1)), hc(n);
    CK(h, cudaMemcpyAsync(hr.data(), dr, sizeof(V) * m, cudaMemcpyDeviceToHost, s));
    CK(h, cudaMemcpyAsync(hc.data(), dc, sizeof(V) * n, cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    h->dr_host.assign(hr.begin(), hr.begin() + m);
    h->dc_host.assign(hc.begin(), hc.end());
    P.sc_x = scx;
    P.sc_y = m > 0 ? scy : nullptr;
    // D-hat of the scaled K
    launch_dhat<V>(h, h->dhat_mode < 0 ? 1 : h->dhat_mode, s);
    CK(h, cudaGetLastError());
    h->pw_base_valid = false;
    h->scaled = true;
    return AAPDHG_OK;
}


}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
// ---------------------------------------------------------------------------
// Checkpoint / resume.  A state blob is a header (the LP's sizes and set-up,
// which must match the handle it is restored into, and the host-side run
// state: steps, primal-weight state, layouts, time used) followed by the
// device arrays in a fixed order: DevState, the iterate pairs, g, D-hat, then
// (when allocated) the two rings and the primal-weight snapshot and base
// D-hat.  Restoring it and iterating gives bit for bit what the run it was
// taken from gives.
// ---------------------------------------------------------------------------
namespace {

constexpr uint64_t STATE_MAGIC = 0x31545354'47445041ull;   // "APDGTST1"

struct StateHeader {
    uint64_t magic;
    int32_t prec, m, n, method, mem, scaled, rings, pw_snap, pw_base, dhat_mode, pad;
    int64_t nnz, N, Npad, pw_period, pw_last_k, bytes;
    LayoutParams lay[2];
    MethodParams mp;
    double pw_gamma, pw_omega, pw_best_kkt, tau_user, sigma_user, time_used;
};

size_t state_bytes(aapdhg_t h) {
    const size_t sv = h->prec == AAPDHG_FP64 ? 8 : 4;
    const bool rings = (h->prec == AAPDHG_FP64 ? (void *)h->pd.DG : (void *)h->pf.DG) != nullptr;
    size_t b = sizeof(StateHeader) + sizeof(DevState) + sv * (size_t)h->N * 4;   // pairs, g, D-hat
    if (rings) b += 2 * sv * (size_t)NSLOT * h->Npad;
    if (h->pw_snap) b += sv * (size_t)h->N;
    if (h->pw_dh_base && h->pw_base_valid) b += sv * (size_t)h->N;
    return b;
}

// The device arrays of the blob, in order: (device pointer, bytes).
template <typename V> std::vector<std::pair<void *, size_t>> state_arrays(aapdhg_t h, bool rings, bool snap,
                                                                            bool base) {
    Prob<V> &P = prob<V>(h);
    const size_t N = (size_t)h->N;
    std::vector<std::pair<void *, size_t>> a;
    a.push_back({h->st, sizeof(DevState)});
    a.push_back({P.UP, sizeof(typename Vec2<V>::T) * N});
    a.push_back({P.g, sizeof(V) * N});
    a.push_back({const_cast<V *>(P.dh), sizeof(V) * N});
    if (rings) {
        a.push_back({P.DG, sizeof(V) * (size_t)NSLOT * h->Npad});
        a.push_back({P.W, sizeof(V) * (size_t)NSLOT * h->Npad});
    }
    if (snap) a.push_back({h->pw_snap, sizeof(V) * N});
    if (base) a.push_back({h->pw_dh_base, sizeof(V) * N});
    return a;
}

template <typename V> aapdhg_status get_state_t(aapdhg_t h, unsigned char *buf) {
    Prob<V> &P = prob<V>(h);
    StateHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    hd.magic = STATE_MAGIC;
    hd.prec = h->prec;
    hd.m = h->m;
    hd.n = h->n;
    hd.method = h->mp.method;
    hd.mem = h->mp.mem;
    hd.scaled = h->scaled ? 1 : 0;
    hd.rings = P.DG ? 1 : 0;
    hd.pw_snap = h->pw_snap ? 1 : 0;
    hd.pw_base = (h->pw_dh_base && h->pw_base_valid) ? 1 : 0;
    hd.dhat_mode = h->dhat_mode;
    hd.nnz = h->nnz;
    hd.N = h->N;
    hd.Npad = h->Npad;
    hd.pw_period = h->pw_period;
    hd.pw_last_k = h->pw_last_k;
    hd.bytes = (int64_t)state_bytes(h);
    hd.lay[0] = h->lay[0];
    hd.lay[1] = h->lay[1];
    hd.mp = h->mp;
    hd.pw_gamma = h->pw_gamma;
    hd.pw_omega = h->pw_omega;
    hd.pw_best_kkt = h->pw_best_kkt;
    hd.tau_user = h->tau_user;
    hd.sigma_user = h->sigma_user;
    hd.time_used = h->time_used;
    std::memcpy(buf, &hd, sizeof(hd));
    size_t off = sizeof(hd);
    for (auto &a : state_arrays<V>(h, hd.rings, hd.pw_snap, hd.pw_base)) {
        CK(h, cudaMemcpyAsync(buf + off, a.first, a.second, cudaMemcpyDeviceToHost, h->stream));
        off += a.second;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    return AAPDHG_OK;
}

template <typename V> aapdhg_status set_state_t(aapdhg_t h, const unsigned char *buf, size_t bytes) {
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (hd.magic != STATE_MAGIC || hd.bytes != (int64_t)bytes)
        return fail(h, AAPDHG_ERR_INVALID, "not a state blob of this library, or truncated");
    if (hd.prec != h->prec || hd.m != h->m || hd.n != h->n || hd.nnz != h->nnz || hd.N != h->N ||
        hd.Npad != h->Npad)
        return fail(h, AAPDHG_ERR_INVALID, "state blob of another LP or precision");
    if (hd.scaled != (h->scaled ? 1 : 0) || hd.method != h->mp.method || hd.mem != h->mp.mem ||
        hd.pw_period != h->pw_period)
        return fail(h, AAPDHG_ERR_INVALID,
                    "state blob taken under another set-up (scaling, method, memory or primal weight period)");
    if (hd.pw_snap && !h->pw_snap) return fail(h, AAPDHG_ERR_INVALID, "state blob needs the primal weight buffers");
    aapdhg_status s;
    if (hd.lay[0].sell_max != h->lay[0].sell_max || hd.lay[0].long_chunk != h->lay[0].long_chunk ||
        hd.lay[1].sell_max != h->lay[1].sell_max || hd.lay[1].long_chunk != h->lay[1].long_chunk) {
        const LayoutParams lay[2] = {hd.lay[0], hd.lay[1]};      // sums in the blob's order
        if ((s = set_layout_t<V>(h, lay)) != AAPDHG_OK) return s;
    }
    if (hd.rings && (s = ensure_rings<V>(h, MAXM)) != AAPDHG_OK) return s;
    if (hd.pw_base && !h->pw_dh_base) return fail(h, AAPDHG_ERR_INVALID, "state blob needs the primal weight buffers");
    size_t off = sizeof(hd);
    for (auto &a : state_arrays<V>(h, hd.rings, hd.pw_snap, hd.pw_base)) {
        CK(h, cudaMemcpyAsync(a.first, buf + off, a.second, cudaMemcpyHostToDevice, h->stream));
        off += a.second;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    h->mp = hd.mp;
    h->have_steps = true;
    h->pw_last_k = hd.pw_last_k;
    h->pw_gamma = hd.pw_gamma;
    h->pw_omega = hd.pw_omega;
    h->pw_best_kkt = hd.pw_best_kkt;
    h->pw_base_valid = hd.pw_base != 0;
    h->tau_user = hd.tau_user;
    h->sigma_user = hd.sigma_user;
    h->time_used = hd.time_used;
    h->dhat_mode = hd.dhat_mode;
    drop_graphs(h);
    return read_state(h);
}

}  // namespace

extern "C" {

aapdhg_status aapdhg_set_allocator(aapdhg_alloc_fn alloc, aapdhg_free_fn free_fn, void *ctx) {
    g_alloc = alloc;
    g_free = free_fn;
    g_ctx = ctx;
    if (!alloc || !free_fn) { g_alloc = nullptr; g_free = nullptr; g_ctx = nullptr; }
    return AAPDHG_OK;
}

aapdhg_status aapdhg_create(int32_t m, int32_t n, int64_t nnz, const int64_t *row_ptr,
                            const int32_t *col_idx, const double *val, const int8_t *row_sense,
                            const double *q, const double *c, const double *lb, const double *ub,
                            int32_t precision, int32_t mem_kind, void *cuda_stream, aapdhg_t *out) {
    NvtxRange range("aapdhg_create");
    if (!out) return fail(nullptr, AAPDHG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (m < 0 || n < 1 || nnz < 0 || nnz >= ((int64_t)1 << 31))
        return fail(nullptr, AAPDHG_ERR_INVALID, "need m >= 0, n >= 1, 0 <= nnz < 2^31");
    if (precision != AAPDHG_FP64 && precision != AAPDHG_MIXED)
        return fail(nullptr, AAPDHG_ERR_INVALID, "unknown precision");
    if (mem_kind != AAPDHG_MEM_HOST && mem_kind != AAPDHG_MEM_DEVICE)
        return fail(nullptr, AAPDHG_ERR_INVALID, "unknown mem_kind");
    if (!row_ptr || (nnz > 0 && (!col_idx || !val)) || (m > 0 && (!row_sense || !q)) || !c || !lb || !ub)
        return fail(nullptr, AAPDHG_ERR_INVALID, "NULL input array");

    // Device inputs are brought to the host once: the renumbering below is host work.
    std::vector<int64_t> rp_h;
    std::vector<int32_t> ci_h;
    std::vector<double> val_h, q_h, c_h, lb_h, ub_h;
    std::vector<int8_t> se_h;
    if (mem_kind == AAPDHG_MEM_DEVICE) {
        rp_h.resize(m + 1); ci_h.resize(nnz); val_h.resize(nnz); q_h.resize(m); se_h.resize(m);
        c_h.resize(n); lb_h.resize(n); ub_h.resize(n);
        cudaError_t e = cudaSuccess;
        auto cp = [&](void *dst, const void *src, size_t b) {
            if (b && e == cudaSuccess) e = cudaMemcpy(dst, src, b, cudaMemcpyDeviceToHost);
        };
        cp(rp_h.data(), row_ptr, 8 * (size_t)(m + 1));
        cp(ci_h.data(), col_idx, 4 * (size_t)nnz);
        cp(val_h.data(), val, 8 * (size_t)nnz);
        cp(q_h.data(), q, 8 * (size_t)m);
        cp(se_h.data(), row_sense, (size_t)m);
        cp(c_h.data(), c, 8 * (size_t)n);
        cp(lb_h.data(), lb, 8 * (size_t)n);
        cp(ub_h.data(), ub, 8 * (size_t)n);
        if (e != cudaSuccess)
            return fail(nullptr, AAPDHG_ERR_CUDA, std::string("reading device inputs: ") + cudaGetErrorString(e));
        row_ptr = rp_h.data(); col_idx = ci_h.data(); val = val_h.data(); q = q_h.data();
        row_sense = se_h.data(); c = c_h.data(); lb = lb_h.data(); ub = ub_h.data();
    }

    {
        const std::string why = validate_lp(m, n, nnz, row_ptr, col_idx, val, row_sense, q, c, lb, ub);
        if (!why.empty()) return fail(nullptr, AAPDHG_ERR_INVALID, why);
    }

    aapdhg_t h = new (std::nothrow) aapdhg_s();
    if (!h) return fail(nullptr, AAPDHG_ERR_OOM, "host allocation");
    h->m = m; h->n = n; h->nnz = nnz; h->N = (int64_t)n + m; h->prec = precision;
    h->Npad = (h->N + 63) & ~(int64_t)63;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) {
        if (cuda_stream) h->stream = (cudaStream_t)cuda_stream;
        else { e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking); h->own_stream = true; }
    }
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->st_host, sizeof(DevState));
    if (e != cudaSuccess) {
        std::string msg = std::string("CUDA setup: ") + cudaGetErrorString(e);
        if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
        delete h;
        return fail(nullptr, AAPDHG_ERR_CUDA, msg);
    }
    h->lo_x.assign(lb, lb + n);
    h->hi_x.assign(ub, ub + n);
    h->sense.assign(row_sense, row_sense + m);

    HostCSR K, KT;
    build_internal(m, n, row_ptr, col_idx, val, h->perm_x, h->perm_y, K, KT);
    aapdhg_status s = precision == AAPDHG_FP64
                          ? setup_device<double>(h, K, KT, row_sense, q, c, lb, ub)
                          : setup_device<float>(h, K, KT, row_sense, q, c, lb, ub);
    if (s == AAPDHG_OK) {
        h->mp.method = AAPDHG_AA; h->mp.mem = 5; h->mp.D = 10.0; h->mp.eps = 1.0;
        h->mp.eta = 1e-10; h->mp.beta = 1.0; h->mp.c_s = 0.2; h->mp.kappa = 1e8; h->mp.c_div = 1.0;
        h->mp.faa_adaptive = 1;
        aapdhg_set_start(h, nullptr, nullptr);
        s = h->sticky;
    }
    if (s != AAPDHG_OK) {
        g_create_err = h->err;
        aapdhg_destroy(h);
        return s;
    }
    *out = h;
    return AAPDHG_OK;
}

aapdhg_status aapdhg_set_steps(aapdhg_t h, double tau, double sigma) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (!(tau > 0) || !(sigma > 0) || !std::isfinite(tau) || !std::isfinite(sigma))
        return fail(h, AAPDHG_ERR_INVALID, "tau and sigma must be finite and > 0");
    h->mp.tau = tau;
    h->tau_user = tau;
    h->sigma_user = sigma;
    h->mp.sigma = sigma;
    h->have_steps = true;
    drop_graphs(h);
    return reset_any(h);
}

aapdhg_status aapdhg_estimate_norm(aapdhg_t h, int32_t iters, uint64_t seed, double *norm) {
    NvtxRange range("aapdhg_estimate_norm");
    if (!h || !norm || iters < 1) return h ? fail(h, AAPDHG_ERR_INVALID, "bad arguments") : AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    return h->prec == AAPDHG_FP64 ? estimate_norm_t<double>(h, iters, seed, norm)
                                  : estimate_norm_t<float>(h, iters, seed, norm);
}

aapdhg_status aapdhg_set_method(aapdhg_t h, int32_t method, int32_t m_A, double D, double eps,
                                double eta, double beta, double c_s, double kappa, double c_div,
                                int32_t dhat_mode, int32_t faa_adaptive) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (method < 0 || method > 2 || m_A < 0 || m_A > AAPDHG_MAX_MEMORY || !(D > 0) || !(eps > 0) ||
        !(eta >= 0) || !(beta > 0 && beta <= 1) || !(c_s > 0 && c_s <= 1) || !(kappa > 0) ||
        !(c_div >= 1) || (dhat_mode != 0 && dhat_mode != 1))
        return fail(h, AAPDHG_ERR_INVALID, "method parameters out of range");
    h->mp.method = method; h->mp.mem = m_A; h->mp.D = D; h->mp.eps = eps; h->mp.eta = eta;
    h->mp.beta = beta; h->mp.c_s = c_s; h->mp.kappa = kappa; h->mp.c_div = c_div;
    h->mp.faa_adaptive = faa_adaptive ? 1 : 0;
    drop_graphs(h);
    // D-hat recomputed on the device when the requested mode differs
    if (dhat_mode != h->dhat_mode) {
        if (h->prec == AAPDHG_FP64) launch_dhat<double>(h, dhat_mode, h->stream);
        else launch_dhat<float>(h, dhat_mode, h->stream);
        CK(h, cudaGetLastError());
        h->dhat_mode = dhat_mode;
        h->pw_base_valid = false;
    }
    return reset_any(h);
}

aapdhg_status aapdhg_set_scaling(aapdhg_t h, int32_t ruiz_iters, int32_t pock_chambolle) {
    NvtxRange range("aapdhg_set_scaling");
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (h->scaled || ruiz_iters < 0 || ruiz_iters > 1000)
        return fail(h, AAPDHG_ERR_INVALID, "scaling is applied at most once, with 0..1000 Ruiz passes");
    drop_graphs(h);
    aapdhg_status s = h->prec == AAPDHG_FP64 ? set_scaling_t<double>(h, ruiz_iters, pock_chambolle)
                                             : set_scaling_t<float>(h, ruiz_iters, pock_chambolle);
    if (s != AAPDHG_OK) return s;
    return reset_any(h);
}

aapdhg_status aapdhg_set_start(aapdhg_t h, const double *x0, const double *y0) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    h->x0.assign(h->n, 0.0);
    h->y0.assign(h->m, 0.0);
    for (int32_t j = 0; j < h->n; ++j) {
        double v = x0 ? x0[j] : 0.0;
        if (!std::isfinite(v)) return fail(h, AAPDHG_ERR_INVALID, "non-finite start");
        h->x0[j] = std::min(std::max(v, h->lo_x[j]), h->hi_x[j]);
    }
    for (int32_t i = 0; i < h->m; ++i) {
        double v = y0 ? y0[i] : 0.0;
        if (!std::isfinite(v)) return fail(h, AAPDHG_ERR_INVALID, "non-finite start");
        if (h->sense[i] == AAPDHG_ROW_GE && v < 0) v = 0;
        h->y0[i] = v;
    }
    return reset_any(h);
}

aapdhg_status aapdhg_reset(aapdhg_t h) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    return reset_any(h);
}

aapdhg_status aapdhg_iterate(aapdhg_t h, int64_t max_iters, double tol, int32_t kkt_every,
                             int64_t *iters_done) {
    NvtxRange range("aapdhg_iterate");
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (!h->have_steps) return fail(h, AAPDHG_ERR_INVALID, "step sizes not set");
    if (max_iters < 0 || std::isnan(tol)) return fail(h, AAPDHG_ERR_INVALID, "bad max_iters or tol");
    return h->prec == AAPDHG_FP64 ? iterate_t<double>(h, max_iters, tol, kkt_every, iters_done)
                                  : iterate_t<float>(h, max_iters, tol, kkt_every, iters_done);
}

aapdhg_status aapdhg_get_iterate(aapdhg_t h, double *x, double *y) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    return h->prec == AAPDHG_FP64 ? get_iterate_t<double>(h, x, y) : get_iterate_t<float>(h, x, y);
}

aapdhg_status aapdhg_set_layout(aapdhg_t h, const int32_t *layout4) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (!layout4) return fail(h, AAPDHG_ERR_INVALID, "layout4 is NULL");
    LayoutParams prm[2];
    for (int w = 0; w < 2; ++w) {
        const int32_t sm = layout4[2 * w], lc = layout4[2 * w + 1];
        if (sm < 1 || sm > 1024 || lc < 32 || lc > (1 << 20) || lc % 32)
            return fail(h, AAPDHG_ERR_INVALID,
                        "layout: 1 <= sell_max <= 1024, long_chunk a multiple of 32 in [32, 2^20]");
        prm[w].sell_max = sm;
        prm[w].long_chunk = lc;
    }
    return h->prec == AAPDHG_FP64 ? set_layout_t<double>(h, prm) : set_layout_t<float>(h, prm);
}

aapdhg_status aapdhg_autotune_layout(aapdhg_t h, int32_t *layout4, double *avg_us) {
    NvtxRange range("aapdhg_autotune_layout");
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    aapdhg_status s = h->prec == AAPDHG_FP64 ? autotune_layout_t<double>(h) : autotune_layout_t<float>(h);
    if (s != AAPDHG_OK) return s;
    if (layout4) {
        layout4[0] = h->lay[0].sell_max;
        layout4[1] = h->lay[0].long_chunk;
        layout4[2] = h->lay[1].sell_max;
        layout4[3] = h->lay[1].long_chunk;
    }
    if (avg_us) for (int k = 0; k < 2 * AAPDHG_LAYOUT_CANDIDATES; ++k) avg_us[k] = h->lay_us[k];
    return AAPDHG_OK;
}

aapdhg_status aapdhg_state_size(aapdhg_t h, size_t *bytes) {
    if (!h || !bytes) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    *bytes = state_bytes(h);
    return AAPDHG_OK;
}

aapdhg_status aapdhg_get_state(aapdhg_t h, void *buf, size_t bytes) {
    NvtxRange range("aapdhg_get_state");
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (!buf || bytes != state_bytes(h))
        return fail(h, AAPDHG_ERR_INVALID, "state buffer is NULL or not aapdhg_state_size bytes");
    return h->prec == AAPDHG_FP64 ? get_state_t<double>(h, (unsigned char *)buf)
                                  : get_state_t<float>(h, (unsigned char *)buf);
}

aapdhg_status aapdhg_set_state(aapdhg_t h, const void *buf, size_t bytes) {
    NvtxRange range("aapdhg_set_state");
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (!buf || bytes < sizeof(StateHeader)) return fail(h, AAPDHG_ERR_INVALID, "state buffer is NULL or too short");
    return h->prec == AAPDHG_FP64 ? set_state_t<double>(h, (const unsigned char *)buf, bytes)
                                  : set_state_t<float>(h, (const unsigned char *)buf, bytes);
}

aapdhg_status aapdhg_set_time_limit(aapdhg_t h, double seconds) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (!(seconds >= 0.0) || std::isinf(seconds))
        return fail(h, AAPDHG_ERR_INVALID, "time limit must be finite and >= 0");
    h->time_limit = seconds;
    return AAPDHG_OK;
}

aapdhg_status aapdhg_get_memory(aapdhg_t h, int32_t capacity, int32_t *count, double *gram,
                                double *rhs, double *dg, double *g) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    return h->prec == AAPDHG_FP64 ? get_memory_t<double>(h, capacity, count, gram, rhs, dg, g)
                                  : get_memory_t<float>(h, capacity, count, gram, rhs, dg, g);
}

aapdhg_status aapdhg_get_kkt(aapdhg_t h, double *out6) {
    if (!h || !out6) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (!h->have_steps) return fail(h, AAPDHG_ERR_INVALID, "step sizes not set");
    return h->prec == AAPDHG_FP64 ? get_kkt_t<double>(h, out6) : get_kkt_t<float>(h, out6);
}

aapdhg_status aapdhg_get_counters(aapdhg_t h, int64_t *aa_steps, int64_t *pdhg_steps,
                                  int64_t *iters, int64_t *ls_failures) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    aapdhg_status s = read_state(h);
    if (s != AAPDHG_OK) return s;
    if (aa_steps) *aa_steps = h->st_host->n_aa;
    if (pdhg_steps) *pdhg_steps = h->st_host->n_pd;
    if (iters) *iters = h->st_host->it;
    if (ls_failures) *ls_failures = h->st_host->n_lsfail;
    return AAPDHG_OK;
}

aapdhg_status aapdhg_set_trace(aapdhg_t h, int64_t capacity) {
    if (!h || capacity < 0) return h ? fail(h, AAPDHG_ERR_INVALID, "capacity < 0") : AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    Trace tr{0, nullptr, nullptr, nullptr, nullptr};
    if (capacity > 0) {
        tr.cap = capacity;
        tr.branch = (int8_t *)dev_alloc(h, capacity);
        tr.gnorm = (double *)dev_alloc(h, 8 * capacity);
        tr.kkt = (double *)dev_alloc(h, 8 * capacity);
        tr.mk = (int32_t *)dev_alloc(h, 4 * capacity);
        if (!tr.branch || !tr.gnorm || !tr.kkt || !tr.mk) return fail(h, AAPDHG_ERR_OOM, "trace buffers");
    }
    h->pf.tr = tr;
    h->pd.tr = tr;
    drop_graphs(h);
    h->tr_cap = capacity;
    return reset_any(h);
}

aapdhg_status aapdhg_get_trace(aapdhg_t h, int64_t *len, int8_t *branch, double *gnorm, double *kkt,
                               int32_t *mk) {
    if (!h || !len) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    const Trace &tr = h->prec == AAPDHG_FP64 ? h->pd.tr : h->pf.tr;
    aapdhg_status s = read_state(h);
    if (s != AAPDHG_OK) return s;
    int64_t n = std::min<int64_t>(*len, std::min<int64_t>(tr.cap, h->st_host->it + 1));
    if (n < 0) n = 0;
    if (n > 0) {
        if (branch) CK(h, cudaMemcpyAsync(branch, tr.branch, n, cudaMemcpyDeviceToHost, h->stream));
        if (gnorm) CK(h, cudaMemcpyAsync(gnorm, tr.gnorm, 8 * n, cudaMemcpyDeviceToHost, h->stream));
        if (kkt) CK(h, cudaMemcpyAsync(kkt, tr.kkt, 8 * n, cudaMemcpyDeviceToHost, h->stream));
        if (mk) CK(h, cudaMemcpyAsync(mk, tr.mk, 4 * n, cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    *len = n;
    return AAPDHG_OK;
}

aapdhg_status aapdhg_profile_kernels(aapdhg_t h, int32_t enable) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    CK(h, cudaStreamSynchronize(h->stream));
    collect_marks(h);
    h->prof_on = enable != 0;
    for (int k = 0; k < NKIND; ++k) { h->prof_ms[k] = 0.0; h->prof_n[k] = 0; }
    return AAPDHG_OK;
}

aapdhg_status aapdhg_get_kernel_profile(aapdhg_t h, int32_t kind, int64_t *launches,
                                        double *total_ms) {
    if (!h || kind < -1 || kind >= NKIND) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    CK(h, cudaStreamSynchronize(h->stream));
    collect_marks(h);
    if (kind == -1) {
        if (launches) *launches = h->launches;
        if (total_ms) *total_ms = 0.0;
    } else {
        if (launches) *launches = h->prof_n[kind];
        if (total_ms) *total_ms = h->prof_ms[kind];
    }
    return AAPDHG_OK;
}

aapdhg_status aapdhg_set_primal_weight(aapdhg_t h, int64_t period, double theta, double eps_zero,
                                       int32_t dhat_blend, double rho_min, double alpha_dec,
                                       double alpha_inc) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (period < 0 || !(theta >= 0 && theta <= 1) || !(eps_zero >= 0) || !std::isfinite(rho_min) ||
        !(alpha_dec >= 0 && alpha_dec <= 1) || !(alpha_inc >= 0 && alpha_inc <= 1))
        return fail(h, AAPDHG_ERR_INVALID, "primal weight parameters out of range");
    h->pw_period = period;
    h->pw_theta = theta;
    h->pw_eps = eps_zero;
    h->pw_dhat = dhat_blend ? 1 : 0;
    h->pw_rho_min = rho_min;
    h->pw_alpha_dec = alpha_dec;
    h->pw_alpha_inc = alpha_inc;
    if (period > 0) {
        const size_t sv = h->prec == AAPDHG_FP64 ? 8 : 4;
        if (!h->pw_snap) h->pw_snap = dev_alloc(h, sv * h->N);
        if (!h->pw_dh_base) {
            h->pw_dh_base = dev_alloc(h, sv * h->N);
            h->pw_base_valid = false;
        }
        if (!h->pw_part) h->pw_part = (double *)dev_alloc(h, sizeof(double) * 2 * h->grid5);
        if (!h->pw_snap || !h->pw_dh_base || !h->pw_part)
            return fail(h, AAPDHG_ERR_OOM, "primal weight buffers");
    } else {
        // back to fixed steps: the given steps and the base D-hat
        h->mp.tau = h->tau_user > 0 ? h->tau_user : h->mp.tau;
        h->mp.sigma = h->sigma_user > 0 ? h->sigma_user : h->mp.sigma;
        if (h->pw_dh_base && h->pw_base_valid) {
            CK(h, cudaMemcpyAsync(h->prec == AAPDHG_FP64 ? (void *)h->pd.dh : (void *)h->pf.dh, h->pw_dh_base,
                                  (h->prec == AAPDHG_FP64 ? 8 : 4) * (size_t)h->N, cudaMemcpyDeviceToDevice,
                                  h->stream));
        }
    }
    drop_graphs(h);
    return reset_any(h);
}

aapdhg_status aapdhg_autotune(aapdhg_t h, int32_t *shape_x, int32_t *shape_y, double *avg_us) {
    NvtxRange range("aapdhg_autotune");
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    aapdhg_status s = h->prec == AAPDHG_FP64 ? autotune_t<double>(h) : autotune_t<float>(h);
    if (s != AAPDHG_OK) return s;
    if (shape_x) *shape_x = h->shape_x;
    if (shape_y) *shape_y = h->shape_y;
    if (avg_us) for (int k = 0; k < 2 * NSHAPE; ++k) avg_us[k] = h->tune_us[k];
    return AAPDHG_OK;
}

aapdhg_status aapdhg_set_task_shape(aapdhg_t h, int32_t shape_x, int32_t shape_y) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (shape_x == -1 && shape_y == -1) {
        h->autotune = true;
        h->tuned = false;
        return AAPDHG_OK;
    }
    if (shape_x < 0 || shape_x >= NSHAPE || shape_y < 0 || shape_y >= NSHAPE)
        return fail(h, AAPDHG_ERR_INVALID, "task shapes are 0 .. AAPDHG_TASK_SHAPES - 1, or both -1");
    h->autotune = false;
    set_shapes(h, shape_x, shape_y);
    drop_graphs(h);
    return AAPDHG_OK;
}

aapdhg_status aapdhg_device_bytes(aapdhg_t h, int64_t *bytes) {
    if (!h || !bytes) return AAPDHG_ERR_INVALID;
    *bytes = h->bytes;
    return AAPDHG_OK;
}

const char *aapdhg_last_error(aapdhg_t h) {
    if (!h) return g_create_err.c_str();
    return h->err.c_str();
}

void aapdhg_destroy(aapdhg_t h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
    drop_graphs(h);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    dev_free_all(h);
    if (h->st_host) cudaFreeHost(h->st_host);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"
