// Host-side pieces shared by the single-LP and the batched runtimes: input
// validation, the longest-first renumbering of K and K', the chunk / SELL-32
// layout of a (possibly block-diagonal) matrix and its upload.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"

namespace aaph {

// NVTX range over a scope (header-only NVTX: free when no tool is attached).
// The API calls and every kernel launch carry one, named by what they do.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Host threads for the set-up work of one LP with `work` entries: 1 below
// 2^20 (thread start-up would dominate), else the hardware's, at most 16.
int host_threads(int64_t work);

// T + 1 ascending cuts of [0, n): equal counts, or equal weight under the
// partial sums prefix[0..n] (a CSR row pointer).
std::vector<int64_t> even_cuts(int64_t n, int T);
template <typename P> std::vector<int64_t> weight_cuts(const P *prefix, int64_t n, int T) {
    std::vector<int64_t> cuts(T + 1, n);
    cuts[0] = 0;
    const double p0 = (double)prefix[0], tot = (double)prefix[n] - p0;
    for (int t = 1; t < T; ++t) {
        const double target = p0 + tot * t / T;
        int64_t lo = cuts[t - 1], hi = n;              // first i with prefix[i] >= target
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if ((double)prefix[mid] < target) lo = mid + 1;
            else hi = mid;
        }
        cuts[t] = lo;
    }
    return cuts;
}

// f(t, lo, hi) for every range t of `cuts`, on one thread each (the calling
// thread takes range 0; a thread that cannot be started runs its range on
// the calling thread).  Each call must write only its own range's outputs.
template <class F> void run_ranges(const std::vector<int64_t> &cuts, F &&f) {
    const int T = (int)cuts.size() - 1;
    std::vector<std::thread> th;
    std::vector<int> inline_t;
    for (int t = 1; t < T; ++t) {
        try {
            th.emplace_back([&f, &cuts, t] { f(t, cuts[t], cuts[t + 1]); });
        } catch (...) {
            inline_t.push_back(t);
        }
    }
    if (T >= 1) f(0, cuts[0], cuts[1]);
    for (int t : inline_t) f(t, cuts[t], cuts[t + 1]);
    for (auto &x : th) x.join();
}

// An allocator whose value-less construction leaves trivial types
// uninitialised: a large host array sized with resize() is first touched by
// the threads that fill it, not zeroed by one thread beforehand.
template <class T> struct uninit_alloc : std::allocator<T> {
    template <class U> struct rebind { typedef uninit_alloc<U> other; };
    uninit_alloc() = default;
    template <class U> uninit_alloc(const uninit_alloc<U> &) noexcept {}
    template <class U> void construct(U *p) noexcept { ::new ((void *)p) U; }
    template <class U, class... A> void construct(U *p, A &&...a) { ::new ((void *)p) U(std::forward<A>(a)...); }
};
template <class T> using hvec = std::vector<T, uninit_alloc<T>>;

struct HostCSR {
    int32_t rows = 0;
    hvec<int32_t> rp, ci;         // every entry written after resize()
    hvec<double> val;
};

// Rows [row0, row0 + rows) of one problem, sorted longest first.
struct RowSeg {
    int32_t row0, rows, pid;
};

// Device-side tables of one matrix built on the host: chunk tables of the long
// rows and the SELL-32 slices of the others.
// Layout parameters: rows longer than sell_max entries are long rows, cut
// into chunks of long_chunk entries (a multiple of 32).
struct LayoutParams {
    int32_t sell_max = aap::SELL_MAX;
    int32_t long_chunk = aap::LONG_CHUNK;
};

// Candidates of the layout tuners (single LP and batch): slice width limit,
// long-row chunk.
constexpr int kNumLayoutCand = 8;
constexpr LayoutParams kLayoutCand[kNumLayoutCand] = {{32, 1024}, {16, 1024}, {64, 1024},  {128, 1024},
                                                      {32, 2048}, {64, 2048}, {128, 2048}, {64, 4096}};

struct LayoutHost {
    int32_t n_long = 0, n_chunks = 0, n_slices = 0;
    int32_t long_chunk = aap::LONG_CHUNK;
    std::vector<int4> chunk_meta;          // (row, long-row id, problem, 0)
    std::vector<int32_t> row_chunk0;       // long-row id -> first chunk
    std::vector<int4> slice_meta;          // (offset, width, first row, rows | problem << 6)
    std::vector<int32_t> sell_ci;
    std::vector<double> sell_val;
};

// Layout of A whose rows form the segments `segs` (each longest first): the
// leading rows of a segment longer than prm.sell_max become long rows, the
// rest slices of up to 32 rows that never cross a segment.  Slices are ordered
// by width, widest first, across all segments (stable, so a single segment
// keeps its row order).  Returns false when the SELL storage would pass 2^31
// entries.
bool build_layout(const HostCSR &A, const std::vector<RowSeg> &segs, LayoutHost &L,
                  const LayoutParams &prm = LayoutParams());

// Internal CSR of K (rows renumbered longest-first, columns mapped to the
// internal variable order) and of K' (likewise), column indices ascending
// within each row.  perm_x / perm_y map internal to caller order.
void build_internal(int32_t m, int32_t n, const int64_t *rp, const int32_t *ci, const double *val,
                    std::vector<int32_t> &perm_x, std::vector<int32_t> &perm_y, HostCSR &K,
                    HostCSR &KT);

// Checks of one LP in the C ABI's input form; returns an empty string when it
// is valid, else the reason.
std::string validate_lp(int32_t m, int32_t n, int64_t nnz, const int64_t *rp, const int32_t *ci,
                        const double *val, const int8_t *sense, const double *q, const double *c,
                        const double *lb, const double *ub);

// Device memory through the allocator installed by aapdhg_set_allocator (or
// cudaMalloc / cudaFree).
void *raw_alloc(size_t bytes);
void raw_free(void *p);

// Upload the layout L of a matrix into `view` (values rounded to V): chunk
// and slice tables, the SELL copy, and the split rows' partial sums and
// counters; `alloc(bytes)` returns tracked device memory.  Synchronises `s`
// (the sources are pageable).
template <typename V, class Alloc>
bool upload_layout(const LayoutHost &L, aap::CSRView<V> &view, Alloc &&alloc, cudaStream_t s) {
    bool ok = true;
    auto put = [&](const auto *src, size_t count) {
        typedef std::remove_cv_t<std::remove_pointer_t<decltype(src)>> T;
        T *d = (T *)alloc(sizeof(T) * std::max<size_t>(count, 1));
        if (!d) { ok = false; return (T *)nullptr; }
        if (count && cudaMemcpyAsync(d, src, sizeof(T) * count, cudaMemcpyHostToDevice, s) != cudaSuccess)
            ok = false;
        return d;
    };
    std::vector<V> sv(L.sell_val.size());
    run_ranges(even_cuts((int64_t)sv.size(), host_threads((int64_t)sv.size())),
               [&](int, int64_t lo, int64_t hi) {
                   for (int64_t i = lo; i < hi; ++i) sv[i] = (V)L.sell_val[i];
               });
    view.n_long = L.n_long;
    view.n_chunks = L.n_chunks;
    view.n_slices = L.n_slices;
    view.long_chunk = L.long_chunk;
    view.chunk_meta = put(L.chunk_meta.data(), L.chunk_meta.size());
    view.row_chunk0 = put(L.row_chunk0.data(), L.row_chunk0.size());
    view.slice_meta = put(L.slice_meta.data(), L.slice_meta.size());
    view.sell_ci = put(L.sell_ci.data(), L.sell_ci.size());
    view.sell_val = put(sv.data(), sv.size());
    view.chunk_part = (V *)alloc(sizeof(V) * 2 * std::max(1, L.n_chunks));
    view.chunk_cnt = (uint32_t *)alloc(sizeof(uint32_t) * std::max(1, L.n_long));
    if (!view.chunk_part || !view.chunk_cnt) ok = false;
    else if (cudaMemsetAsync(view.chunk_cnt, 0, sizeof(uint32_t) * std::max(1, L.n_long), s) != cudaSuccess)
        ok = false;
    if (cudaStreamSynchronize(s) != cudaSuccess) ok = false;
    return ok;
}

// Upload A's CSR (values rounded to V) into `view`.
template <typename V, class Alloc>
bool upload_matrix(const HostCSR &A, aap::CSRView<V> &view, Alloc &&alloc, cudaStream_t s) {
    bool ok = true;
    auto put = [&](const auto *src, size_t count) {
        typedef std::remove_cv_t<std::remove_pointer_t<decltype(src)>> T;
        T *d = (T *)alloc(sizeof(T) * std::max<size_t>(count, 1));
        if (!d) { ok = false; return (T *)nullptr; }
        if (count && cudaMemcpyAsync(d, src, sizeof(T) * count, cudaMemcpyHostToDevice, s) != cudaSuccess)
            ok = false;
        return d;
    };
    std::vector<V> v(A.val.size());
    run_ranges(even_cuts((int64_t)v.size(), host_threads((int64_t)v.size())),
               [&](int, int64_t lo, int64_t hi) {
                   for (int64_t i = lo; i < hi; ++i) v[i] = (V)A.val[i];
               });
    view.rows = A.rows;
    view.rp = put(A.rp.data(), A.rp.size());
    view.ci = put(A.ci.data(), A.ci.size());
    view.val = put(v.data(), v.size());
    if (cudaStreamSynchronize(s) != cudaSuccess) ok = false;
    return ok;
}

// Upload A (its CSR, values rounded to V) and its layout into `view`.
template <typename V, class Alloc>
bool upload_csr(const HostCSR &A, const LayoutHost &L, aap::CSRView<V> &view, Alloc &&alloc,
                cudaStream_t s) {
    const bool a = upload_matrix<V>(A, view, alloc, s);
    const bool b = upload_layout<V>(L, view, alloc, s);
    return a && b;
}
}  // namespace aaph
