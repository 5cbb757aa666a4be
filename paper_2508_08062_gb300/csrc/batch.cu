// Host runtime and C ABI of the batched solver (aapdhg_batch_*): many
// independent LPs packed into one block-diagonal LP and advanced together by
// the kernels of batch.cuh.
//
// create():  validate every LP, renumber each one's rows and columns
//            longest-first (as the single-LP solver does), pad its variable
//            and constraint ranges to multiples of 4, pack K and K' of all
//            problems into one matrix each (SELL slices of all problems
//            ordered by width), cut each problem's elements into chunks for
//            the per-problem reductions, and move everything to the device.
// iterate(): the kernel sequence of one batch iteration, in CUDA graphs of
//            CHUNK_ITERS iterations; once per chunk the host reads the
//            per-problem state headers (one strided copy) and stops when every
//            problem has met the tolerance or failed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/aapdhg.h"
#include "batch.cuh"
#include "host.h"
#include "precond.cuh"

using namespace aap;
using namespace aaph;

namespace {

constexpr int B_CHUNK_ITERS = 64;
thread_local std::string g_batch_create_err;

// Per-problem header read by the host each chunk: it, n_aa, n_pd, n_lsfail,
// done, error, init_done (the leading fields of DevState), 8-byte aligned.
constexpr size_t HDR = (offsetof(DevState, want_aa) + 7) & ~(size_t)7;

enum { BK_XSTEP = 0, BK_YSTEP = 1, BK_MEMORY = 2, BK_MIX = 3, BK_KKT = 4, BK_GRAM = 5, BK_N = 6 };

}  // namespace

struct aapdhg_batch_s {
    int32_t nprob = 0;
    int32_t prec = AAPDHG_MIXED;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0, sm_count = 0;
    aapdhg_status sticky = AAPDHG_OK;
    std::string err;
    struct Alloc { void *p; size_t bytes; };
    std::vector<Alloc> allocs;
    int64_t bytes = 0;

    // problem p: caller sizes, padded sizes, offsets of its variables and
    // constraints in the packed order, and its renumbering (internal -> caller)
    std::vector<int32_t> m, n, nxp, nyp;
    std::vector<int64_t> xoff, yoff, xcat, ycat;   // packed offsets; offsets into caller arrays
    std::vector<int32_t> perm_x, perm_y;           // concatenated, local indices
    std::vector<double> lo_x, hi_x, x0, y0;        // caller order, concatenated
    std::vector<int8_t> sense;
    std::vector<double> tau, sigma;
    std::vector<float> tau_f, sigma_f;             // the steps rounded once (mixed precision)
    int64_t n_tot = 0, m_tot = 0, N = 0, Npad = 0;

    Prob<float> pf{};
    Prob<double> pd{};
    BatchView<float> bf{};
    BatchView<double> bd{};
    MethodParams mp{};
    DevState *stb = nullptr;
    double *ptol_dev = nullptr;                    // per-problem tolerances (when set)
    unsigned char *hdr_host = nullptr;             // pinned: nprob headers
    int64_t g = 0;                                 // batch iterations launched (the start one included)
    int32_t kkt_every = 0;
    int32_t dhat_mode = -1;
    bool scaled = false;
    std::vector<double> dr, dc;                    // Dr (m_tot), Dc (n_tot) in packed order
    bool have_rings = false;
    // CUDA graphs of full chunks keyed by (KKT phase, parity, kkt_every, tol)
    cudaStream_t cap_stream = nullptr;
    struct GraphEntry { cudaGraphExec_t exec; int64_t phase; int parity; int32_t kkt_every; double tol; };
    std::vector<GraphEntry> graphs;
    bool use_graphs = true;
    // task shapes of the two half-step kernels (autotuned at the first iterate)
    int32_t shape_x = 0, shape_y = 0;
    bool tuned = false, autotune = true;
    int32_t gridx[NSHAPE] = {}, gridy[NSHAPE] = {};
    double tune_us[2 * NSHAPE] = {};
    // layouts of the packed K' and K (slice width limit, long-row chunk), the
    // problems' row segments they are built from, and the device allocations
    // of their layout parts, by matrix (0: K', 1: K)
    LayoutParams lay[2];
    std::vector<RowSeg> segs[2];
    std::vector<void *> lay_ptrs[2];
    double lay_us[2 * kNumLayoutCand] = {};
    int64_t nnz_tot = 0;
    // primal weight update (off when pw_period = 0): per problem gamma, omega
    // and the lowest KKT at an update point (pw_w), the blend weight and
    // update flag of the last try, the snapshot
    // of u at the last update point, the base D-hat
    int64_t pw_period = 0, pw_last_g = -1;
    PwParams pw{0.5, 1e-10, 0.1, 0.1, 0.9};
    int32_t pw_dhat = 1;
    void *pw_snap = nullptr, *pw_dh_base = nullptr;
    double *pw_part = nullptr, *pw_w = nullptr, *pw_alpha = nullptr;
    int32_t *pw_upd = nullptr;
    bool pw_base_valid = false;            // pw_dh_base holds the current base D-hat
    // instrumentation
    bool prof_on = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_kind;
    double prof_ms[BK_N] = {0, 0, 0, 0, 0, 0};
    int64_t prof_n[BK_N] = {0, 0, 0, 0, 0, 0};
    int64_t launches = 0;
};

typedef aapdhg_batch_s *bh_t;

namespace {

aapdhg_status bfail(bh_t h, aapdhg_status s, const std::string &msg) {
    if (h) {
        if (h->sticky == AAPDHG_OK) {
            h->sticky = s;
            h->err = msg;
        }
    } else {
        g_batch_create_err = msg;
    }
    return s;
}

#define BCK(h, call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bfail((h), AAPDHG_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void *bdev_alloc(bh_t h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void *p = raw_alloc(bytes);
    if (p) {
        h->allocs.push_back({p, bytes});
        h->bytes += (int64_t)bytes;
    }
    return p;
}

template <typename T> T *bput(bh_t h, const std::vector<T> &src, bool *ok) {
    T *d = (T *)bdev_alloc(h, sizeof(T) * std::max<size_t>(src.size(), 1));
    if (!d) { *ok = false; return nullptr; }
    if (!src.empty() &&
        cudaMemcpyAsync(d, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        *ok = false;
    return d;
}

template <typename V> Prob<V> &bprob(bh_t h);
template <> Prob<float> &bprob<float>(bh_t h) { return h->pf; }
template <> Prob<double> &bprob<double>(bh_t h) { return h->pd; }
template <typename V> BatchView<V> &bview(bh_t h);
template <> BatchView<float> &bview<float>(bh_t h) { return h->bf; }
template <> BatchView<double> &bview<double>(bh_t h) { return h->bd; }

int bgrid(bh_t h, int64_t need, int occ) {
    const int64_t cap = (int64_t)h->sm_count * std::max(occ, 1);
    return (int)std::max<int64_t>(1, std::min<int64_t>(need, cap));
}

template <class K> int boccupancy(K kernel) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, BLOCK, 0) != cudaSuccess) {
        cudaGetLastError();
        occ = 1;
    }
    return std::max(occ, 1);
}

const char *const kBKindName[BK_N] = {"aapdhg batch x-step", "aapdhg batch y-step", "aapdhg batch memory pass",
                                      "aapdhg batch AA mix", "aapdhg batch KKT", "aapdhg batch Gram pass"};

void bmark_begin(bh_t h, int kind) {
    h->launches += 1;
    nvtxRangePushA(kBKindName[kind]);
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

void bmark_end(bh_t h) {
    nvtxRangePop();
    if (!h->prof_on || h->ev_kind.empty()) return;
    cudaEventRecord(h->ev[2 * h->ev_kind.size() - 1], h->stream);
}

void bcollect(bh_t h) {
    for (size_t i = 0; i < h->ev_kind.size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]) == cudaSuccess) {
            h->prof_ms[h->ev_kind[i]] += ms;
            h->prof_n[h->ev_kind[i]] += 1;
        }
    }
    h->ev_kind.clear();
}

void bdrop_graphs(bh_t h) {
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
}

// ---------------------------------------------------------------------------
// set-up
// ---------------------------------------------------------------------------
// Grids per task shape for the common (non-KKT) half-step variants: all their
// blocks resident.
template <typename V> void bhalf_step_grids(bh_t h) {
    Prob<V> &P = bprob<V>(h);
    const int occx[NSHAPE] = {boccupancy(k_xstep_b<V, false, 0>), boccupancy(k_xstep_b<V, false, 1>),
                              boccupancy(k_xstep_b<V, false, 2>), boccupancy(k_xstep_b<V, false, 3>),
                              boccupancy(k_xstep_b<V, false, 4>)};
    const int occy[NSHAPE] = {boccupancy(k_ystep_b<V, false, 0>), boccupancy(k_ystep_b<V, false, 1>),
                              boccupancy(k_ystep_b<V, false, 2>), boccupancy(k_ystep_b<V, false, 3>),
                              boccupancy(k_ystep_b<V, false, 4>)};
    for (int sh = 0; sh < NSHAPE; ++sh) {
        const int g = task_shape(sh).g;
        h->gridx[sh] = bgrid(h, (P.KT.ntasks(g) + WARPS - 1) / WARPS, occx[sh]);
        h->gridy[sh] = bgrid(h, (P.K.ntasks(g) + WARPS - 1) / WARPS, occy[sh]);
    }
}

template <typename V>
aapdhg_status bsetup(bh_t h, const HostCSR &K, const HostCSR &KT, const std::vector<RowSeg> &segK,
                     const std::vector<RowSeg> &segKT, const std::vector<double> &cv,
                     const std::vector<double> &qv, const std::vector<double> &lov,
                     const std::vector<double> &hiv, const std::vector<double> &pnorm) {
    typedef typename Vec2<V>::T V2;
    Prob<V> &P = bprob<V>(h);
    BatchView<V> &B = bview<V>(h);
    bool ok = true;
    P.m = (int32_t)h->m_tot;
    P.n = (int32_t)h->n_tot;
    P.N = h->N;
    P.Npad = h->Npad;
    auto alloc = [&](size_t b) { return bdev_alloc(h, b); };
    h->segs[0] = segKT;
    h->segs[1] = segK;
    h->nnz_tot = (int64_t)K.ci.size();
    for (int which = 0; which < 2 && ok; ++which) {
        LayoutHost L;
        const HostCSR &A = which ? K : KT;
        if (!build_layout(A, h->segs[which], L, h->lay[which]))
            return bfail(h, AAPDHG_ERR_INVALID, "packed SELL storage exceeds 2^31 entries");
        CSRView<V> &view = which ? P.K : P.KT;
        if (!upload_matrix<V>(A, view, alloc, h->stream)) ok = false;
        std::vector<void *> &rec = h->lay_ptrs[which];
        auto track = [&](size_t b) {
            void *q = bdev_alloc(h, b);
            if (q) rec.push_back(q);
            return q;
        };
        if (!upload_layout<V>(L, view, track, h->stream)) ok = false;
    }
    auto to_v = [](const std::vector<double> &a) {
        std::vector<V> o(a.size());
        for (size_t i = 0; i < a.size(); ++i) o[i] = (V)a[i];
        return o;
    };
    P.c = bput(h, to_v(cv), &ok);
    P.q = bput(h, to_v(qv), &ok);
    P.lo = bput(h, to_v(lov), &ok);
    P.hi = bput(h, to_v(hiv), &ok);
    P.UP = (V2 *)bdev_alloc(h, sizeof(V2) * h->N);
    P.dh = (V *)bdev_alloc(h, sizeof(V) * h->N);
    P.g = (V *)bdev_alloc(h, sizeof(V) * h->N);
    P.DG = P.W = nullptr;
    P.sc_x = P.sc_y = nullptr;
    P.part1 = P.part2 = P.part3 = nullptr;
    P.tr = Trace{0, nullptr, nullptr, nullptr, nullptr};
    P.st = nullptr;
    if (!P.UP || !P.dh || !P.g) ok = false;
    bhalf_step_grids<V>(h);
    P.grid1 = h->gridx[0];
    P.grid2 = h->gridy[0];

    // chunks of every problem's elements: its variables, then its constraints
    std::vector<int4> chunk;
    std::vector<int32_t> pchunk0(h->nprob + 1, 0);
    for (int32_t p = 0; p < h->nprob; ++p) {
        pchunk0[p] = (int32_t)chunk.size();
        for (int part = 0; part < 2; ++part) {
            const int64_t base = part ? h->n_tot + h->yoff[p] : h->xoff[p];
            const int64_t len = part ? h->nyp[p] : h->nxp[p];
            for (int64_t e = 0; e < len; e += BCHUNK)
                chunk.push_back(make_int4(p, (int32_t)(base + e), (int32_t)std::min<int64_t>(BCHUNK, len - e), part));
        }
    }
    pchunk0[h->nprob] = (int32_t)chunk.size();
    B.nprob = h->nprob;
    B.n_tot = h->n_tot;
    B.m_tot = h->m_tot;
    if (chunk.size() > 65535)                // the Gram pass's grid has one row of blocks per chunk
        return bfail(h, AAPDHG_ERR_INVALID, "batch too large: more than 65535 element chunks of 8192");
    B.nchunk = (int32_t)chunk.size();
    B.chunk = bput(h, chunk, &ok);
    B.pchunk0 = bput(h, pchunk0, &ok);
    B.pnorm = bput(h, pnorm, &ok);
    B.tau = (const double *)bdev_alloc(h, sizeof(double) * h->nprob);
    B.sigma = (const double *)bdev_alloc(h, sizeof(double) * h->nprob);
    B.tau_v = (const V *)bdev_alloc(h, sizeof(V) * h->nprob);
    B.sigma_v = (const V *)bdev_alloc(h, sizeof(V) * h->nprob);
    B.stb = (DevState *)bdev_alloc(h, sizeof(DevState) * h->nprob);
    B.kterm = (V *)bdev_alloc(h, sizeof(V) * (3 * h->n_tot + 2 * h->m_tot));
    B.cpart = (double *)bdev_alloc(h, sizeof(double) * NBV * B.nchunk);
    B.pcnt = (uint32_t *)bdev_alloc(h, sizeof(uint32_t) * h->nprob);
    if (!B.tau || !B.sigma || !B.tau_v || !B.sigma_v || !B.stb || !B.kterm || !B.cpart || !B.pcnt) ok = false;
    if (!ok) return bfail(h, AAPDHG_ERR_OOM, "device allocation or copy failed during create");
    h->stb = B.stb;
    BCK(h, cudaMemsetAsync(B.stb, 0, sizeof(DevState) * h->nprob, h->stream));
    BCK(h, cudaMemsetAsync(B.pcnt, 0, sizeof(uint32_t) * h->nprob, h->stream));
    BCK(h, cudaMemsetAsync(B.kterm, 0, sizeof(V) * (3 * h->n_tot + 2 * h->m_tot), h->stream));
    k_dhat<V><<<bgrid(h, (h->N + WARPS - 1) / WARPS, 8), BLOCK, 0, h->stream>>>(
        P.KT, P.K, P.n, P.m, 1, const_cast<V *>(P.dh));
    BCK(h, cudaGetLastError());
    h->dhat_mode = 1;
    BCK(h, cudaStreamSynchronize(h->stream));
    return AAPDHG_OK;
}

template <typename V> aapdhg_status bensure_rings(bh_t h) {
    Prob<V> &P = bprob<V>(h);
    if (h->have_rings) return AAPDHG_OK;
    P.DG = (V *)bdev_alloc(h, sizeof(V) * (size_t)NSLOT * h->Npad);
    P.W = (V *)bdev_alloc(h, sizeof(V) * (size_t)NSLOT * h->Npad);
    BatchView<V> &B = bview<V>(h);
    B.gpart = (double *)bdev_alloc(h, sizeof(double) * (size_t)GRAM_MAXPAIRS * B.nchunk);
    if (!P.DG || !P.W || !B.gpart)
        return bfail(h, AAPDHG_ERR_OOM, "device allocation of the Anderson memory failed");
    h->have_rings = true;
    return AAPDHG_OK;
}

// The given steps of every problem into the device arrays (FP64 and the
// iterate precision).
aapdhg_status bupload_steps(bh_t h) {
    const double *dt = h->prec == AAPDHG_FP64 ? h->bd.tau : h->bf.tau;
    const double *ds = h->prec == AAPDHG_FP64 ? h->bd.sigma : h->bf.sigma;
    BCK(h, cudaMemcpyAsync(const_cast<double *>(dt), h->tau.data(), 8 * (size_t)h->nprob, cudaMemcpyHostToDevice,
                           h->stream));
    BCK(h, cudaMemcpyAsync(const_cast<double *>(ds), h->sigma.data(), 8 * (size_t)h->nprob,
                           cudaMemcpyHostToDevice, h->stream));
    if (h->prec == AAPDHG_FP64) {
        BCK(h, cudaMemcpyAsync(const_cast<double *>(h->bd.tau_v), h->tau.data(), 8 * (size_t)h->nprob,
                               cudaMemcpyHostToDevice, h->stream));
        BCK(h, cudaMemcpyAsync(const_cast<double *>(h->bd.sigma_v), h->sigma.data(), 8 * (size_t)h->nprob,
                               cudaMemcpyHostToDevice, h->stream));
    } else {
        h->tau_f.assign(h->tau.begin(), h->tau.end());
        h->sigma_f.assign(h->sigma.begin(), h->sigma.end());
        BCK(h, cudaMemcpyAsync(const_cast<float *>(h->bf.tau_v), h->tau_f.data(), 4 * (size_t)h->nprob,
                               cudaMemcpyHostToDevice, h->stream));
        BCK(h, cudaMemcpyAsync(const_cast<float *>(h->bf.sigma_v), h->sigma_f.data(), 4 * (size_t)h->nprob,
                               cudaMemcpyHostToDevice, h->stream));
    }
    return AAPDHG_OK;
}

// Start of every problem: u^0 (projected start, scaled when the LP is) in
// component 0, state cleared, batch counter at 0.
template <typename V> aapdhg_status breset(bh_t h) {
    typedef typename Vec2<V>::T V2;
    Prob<V> &P = bprob<V>(h);
    std::vector<V2> up(h->N);
    for (auto &e : up) { e.x = V(0); e.y = V(0); }
    for (int32_t p = 0; p < h->nprob; ++p) {
        const int32_t *px = h->perm_x.data() + h->xcat[p];
        const int32_t *py = h->perm_y.data() + h->ycat[p];
        for (int32_t j = 0; j < h->n[p]; ++j) {
            const int64_t e = h->xoff[p] + j;
            const double v = h->x0[h->xcat[p] + px[j]];
            up[e].x = (V)(h->scaled ? v / h->dc[e] : v);
        }
        for (int32_t i = 0; i < h->m[p]; ++i) {
            const int64_t r = h->yoff[p] + i;
            const double v = h->y0[h->ycat[p] + py[i]];
            up[h->n_tot + r].x = (V)(h->scaled ? v / h->dr[r] : v);
        }
    }
    BCK(h, cudaMemcpyAsync(P.UP, up.data(), sizeof(V2) * h->N, cudaMemcpyHostToDevice, h->stream));
    BCK(h, cudaMemsetAsync(h->stb, 0, sizeof(DevState) * h->nprob, h->stream));
    if (h->pw_period > 0) {
        // a run starts with the given steps, omega^0 = sqrt(sigma / tau),
        // gamma = sqrt(tau sigma) and the base D-hat (R13)
        aapdhg_status s = bupload_steps(h);
        if (s != AAPDHG_OK) return s;
        std::vector<double> w(3 * (size_t)h->nprob);
        for (int32_t p = 0; p < h->nprob; ++p) {
            const double t = h->tau[p], sg = h->sigma[p];
            w[3 * p] = t > 0 ? sqrt(t * sg) : 0.0;
            w[3 * p + 1] = t > 0 ? sqrt(sg / t) : 1.0;
            w[3 * p + 2] = INFINITY;
        }
        BCK(h, cudaMemcpyAsync(h->pw_w, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice, h->stream));
        V *dh = const_cast<V *>(P.dh);
        if (!h->pw_base_valid) {
            BCK(h, cudaMemcpyAsync(h->pw_dh_base, dh, sizeof(V) * h->N, cudaMemcpyDeviceToDevice, h->stream));
            h->pw_base_valid = true;
        } else {
            BCK(h, cudaMemcpyAsync(dh, h->pw_dh_base, sizeof(V) * h->N, cudaMemcpyDeviceToDevice, h->stream));
        }
        h->pw_last_g = -1;
    }
    BCK(h, cudaStreamSynchronize(h->stream));
    h->g = 0;
    return AAPDHG_OK;
}

aapdhg_status breset_any(bh_t h) { return h->prec == AAPDHG_FP64 ? breset<double>(h) : breset<float>(h); }

// ---------------------------------------------------------------------------
// one batch iteration
// ---------------------------------------------------------------------------
template <typename V, int MC> void blaunch_memory_mix(bh_t h, int cur) {
    Prob<V> &P = bprob<V>(h);
    BatchView<V> &B = bview<V>(h);
    const int M = (h->mp.method == 0) ? 0 : h->mp.mem;
    const int fp64 = h->prec == AAPDHG_FP64 ? 1 : 0;
    bmark_begin(h, BK_MEMORY);
    k_memory_b<V><<<B.nchunk, BLOCK, 0, h->stream>>>(P, B, h->mp, cur);
    bmark_end(h);
    bmark_begin(h, BK_GRAM);             // the push, and the Gram pass of the attempts
    k_gram_b<<<h->nprob, 32, 0, h->stream>>>(h->bf, h->bd, fp64, h->mp);
    if (M > 0) {
        k_gram_cols_b<V><<<dim3(M, B.nchunk), BLOCK, 0, h->stream>>>(P, B);
        k_solve_b<<<h->nprob, 32, 0, h->stream>>>(h->bf, h->bd, fp64, h->mp);
        h->launches += 2;
    }
    bmark_end(h);
    if (M > 0) {
        bmark_begin(h, BK_MIX);
        k_mix_b<V, MC><<<B.nchunk, BLOCK, 0, h->stream>>>(P, B, h->mp, cur);
        bmark_end(h);
    }
}

template <typename V, bool KKT> void blaunch_x(bh_t h, int shape, int cur, int mode) {
    Prob<V> &P = bprob<V>(h);
    BatchView<V> &B = bview<V>(h);
    if (shape == 1) k_xstep_b<V, KKT, 1><<<P.grid1, BLOCK, 0, h->stream>>>(P, B, cur, mode);
    else if (shape == 2) k_xstep_b<V, KKT, 2><<<P.grid1, BLOCK, 0, h->stream>>>(P, B, cur, mode);
    else if (shape == 3) k_xstep_b<V, KKT, 3><<<P.grid1, BLOCK, 0, h->stream>>>(P, B, cur, mode);
    else if (shape == 4) k_xstep_b<V, KKT, 4><<<P.grid1, BLOCK, 0, h->stream>>>(P, B, cur, mode);
    else k_xstep_b<V, KKT, 0><<<P.grid1, BLOCK, 0, h->stream>>>(P, B, cur, mode);
}

template <typename V, bool KKT> void blaunch_y(bh_t h, int shape, int cur, int mode) {
    Prob<V> &P = bprob<V>(h);
    BatchView<V> &B = bview<V>(h);
    if (shape == 1) k_ystep_b<V, KKT, 1><<<P.grid2, BLOCK, 0, h->stream>>>(P, B, cur, mode);
    else if (shape == 2) k_ystep_b<V, KKT, 2><<<P.grid2, BLOCK, 0, h->stream>>>(P, B, cur, mode);
    else if (shape == 3) k_ystep_b<V, KKT, 3><<<P.grid2, BLOCK, 0, h->stream>>>(P, B, cur, mode);
    else if (shape == 4) k_ystep_b<V, KKT, 4><<<P.grid2, BLOCK, 0, h->stream>>>(P, B, cur, mode);
    else k_ystep_b<V, KKT, 0><<<P.grid2, BLOCK, 0, h->stream>>>(P, B, cur, mode);
}

void bset_shapes(bh_t h, int sx, int sy) {
    h->shape_x = sx;
    h->shape_y = sy;
    h->pf.grid1 = h->pd.grid1 = h->gridx[sx];
    h->pf.grid2 = h->pd.grid2 = h->gridy[sy];
}

// Autotuning of the two half-step kernels, as for the single-LP solver: every
// task shape timed on the packed matrices (timing mode: no run state changes).
template <typename V> aapdhg_status bautotune(bh_t h) {
    Prob<V> &P = bprob<V>(h);
    const int cur = (int)(h->g & 1);
    cudaEvent_t e0, e1;
    BCK(h, cudaEventCreate(&e0));
    BCK(h, cudaEventCreate(&e1));
    // two interleaved rounds, the faster of the two kept per shape (robust to
    // clock ramps and to whatever ran just before)
    double tx[NSHAPE], ty[NSHAPE];
    for (int sh = 0; sh < NSHAPE; ++sh) tx[sh] = ty[sh] = 1e30;
    for (int round = 0; round < 2; ++round)
        for (int sh = 0; sh < NSHAPE; ++sh) {
            P.grid1 = h->gridx[sh];
            P.grid2 = h->gridy[sh];
            float ms = 0.f;
            for (int w = 0; w < 2; ++w) blaunch_x<V, false>(h, sh, cur, MODE_TUNE);
            cudaEventRecord(e0, h->stream);
            for (int r = 0; r < 5; ++r) blaunch_x<V, false>(h, sh, cur, MODE_TUNE);
            cudaEventRecord(e1, h->stream);
            BCK(h, cudaEventSynchronize(e1));
            cudaEventElapsedTime(&ms, e0, e1);
            tx[sh] = std::min(tx[sh], 1e3 * ms / 5);
            for (int w = 0; w < 2; ++w) blaunch_y<V, false>(h, sh, cur, MODE_TUNE);
            cudaEventRecord(e0, h->stream);
            for (int r = 0; r < 5; ++r) blaunch_y<V, false>(h, sh, cur, MODE_TUNE);
            cudaEventRecord(e1, h->stream);
            BCK(h, cudaEventSynchronize(e1));
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
    BCK(h, cudaGetLastError());
    bset_shapes(h, bx, by);
    h->tuned = true;
    bdrop_graphs(h);
    return AAPDHG_OK;
}

// ---------------------------------------------------------------------------
// Layouts of the packed K' and K (slice width limit, long-row chunk), rebuilt
// from the matrices on the device with every problem's own row segments, as
// the single-LP runtime does.  A problem's rows never share a slice with
// another problem's, so each problem's sums depend on the layout parameters
// only.  The run state is kept; the task shapes are tuned again.
// ---------------------------------------------------------------------------
void bdev_free_ptrs(bh_t h, const std::vector<void *> &ptrs) {
    for (void *q : ptrs)
        for (size_t i = 0; i < h->allocs.size(); ++i)
            if (h->allocs[i].p == q) {
                h->bytes -= (int64_t)h->allocs[i].bytes;
                raw_free(q);
                h->allocs.erase(h->allocs.begin() + (long)i);
                break;
            }
}

template <typename V> aapdhg_status bdownload_csr(bh_t h, const CSRView<V> &v, int64_t nnz, HostCSR &A) {
    A.rows = v.rows;
    A.rp.resize((size_t)v.rows + 1);
    A.ci.resize((size_t)nnz);
    A.val.resize((size_t)nnz);
    std::vector<V> tmp((size_t)std::max<int64_t>(nnz, 1));
    BCK(h, cudaMemcpyAsync(A.rp.data(), v.rp, sizeof(int32_t) * ((size_t)v.rows + 1), cudaMemcpyDeviceToHost,
                           h->stream));
    if (nnz > 0) {
        BCK(h, cudaMemcpyAsync(A.ci.data(), v.ci, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToHost, h->stream));
        BCK(h, cudaMemcpyAsync(tmp.data(), v.val, sizeof(V) * (size_t)nnz, cudaMemcpyDeviceToHost, h->stream));
    }
    BCK(h, cudaStreamSynchronize(h->stream));
    for (int64_t k = 0; k < nnz; ++k) A.val[k] = (double)tmp[k];
    return AAPDHG_OK;
}

template <typename V> aapdhg_status bset_layout_t(bh_t h, const LayoutParams (&prm)[2]) {
    Prob<V> &P = bprob<V>(h);
    BCK(h, cudaStreamSynchronize(h->stream));
    CSRView<V> nv[2] = {P.KT, P.K};
    std::vector<void *> rec[2];
    bool ok = true;
    for (int w = 0; w < 2 && ok; ++w) {
        HostCSR A;
        aapdhg_status s = bdownload_csr<V>(h, nv[w], h->nnz_tot, A);
        if (s != AAPDHG_OK) return s;
        LayoutHost L;
        if (!build_layout(A, h->segs[w], L, prm[w])) {
            bdev_free_ptrs(h, rec[0]);
            return bfail(h, AAPDHG_ERR_INVALID, "packed SELL storage exceeds 2^31 entries");
        }
        auto track = [&](size_t b) {
            void *q = bdev_alloc(h, b);
            if (q) rec[w].push_back(q);
            return q;
        };
        if (!upload_layout<V>(L, nv[w], track, h->stream)) ok = false;
    }
    if (!ok) {
        bdev_free_ptrs(h, rec[0]);
        bdev_free_ptrs(h, rec[1]);
        return bfail(h, AAPDHG_ERR_OOM, "layout: device allocation or copy failed");
    }
    bdev_free_ptrs(h, h->lay_ptrs[0]);
    bdev_free_ptrs(h, h->lay_ptrs[1]);
    h->lay_ptrs[0] = rec[0];
    h->lay_ptrs[1] = rec[1];
    P.KT = nv[0];
    P.K = nv[1];
    h->lay[0] = prm[0];
    h->lay[1] = prm[1];
    bhalf_step_grids<V>(h);
    bset_shapes(h, 0, 0);
    h->tuned = false;
    bdrop_graphs(h);
    return AAPDHG_OK;
}

// Every candidate layout for both matrices, with the task shapes tuned on it;
// K' keeps the candidate with the fastest x-step, K the one with the fastest
// y-step.
template <typename V> aapdhg_status bautotune_layout_t(bh_t h) {
    double bestx = INFINITY, besty = INFINITY;
    int bx_i = 0, by_i = 0;
    for (int c = 0; c < kNumLayoutCand; ++c) {
        const LayoutParams both[2] = {kLayoutCand[c], kLayoutCand[c]};
        aapdhg_status s = bset_layout_t<V>(h, both);
        if (s == AAPDHG_OK) s = bautotune<V>(h);
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
    aapdhg_status s = bset_layout_t<V>(h, chosen);
    if (s == AAPDHG_OK) s = bautotune<V>(h);
    return s;
}

template <typename V> void blaunch_iteration(bh_t h, int64_t g, int mode) {
    BatchView<V> &B = bview<V>(h);
    const int cur = (int)(g & 1);
    const bool kkt = mode == MODE_EVAL || (h->kkt_every > 0 && g >= 1 && (g - 1) % h->kkt_every == 0);
    bmark_begin(h, BK_XSTEP);
    if (kkt) blaunch_x<V, true>(h, h->shape_x, cur, mode);
    else blaunch_x<V, false>(h, h->shape_x, cur, mode);
    bmark_end(h);
    bmark_begin(h, BK_YSTEP);
    if (kkt) blaunch_y<V, true>(h, h->shape_y, cur, mode);
    else blaunch_y<V, false>(h, h->shape_y, cur, mode);
    bmark_end(h);
    if (kkt) {
        bmark_begin(h, BK_KKT);
        k_kkt_b<V><<<B.nchunk, BLOCK, 0, h->stream>>>(B, h->mp.tol, mode);   // ptol overrides tol
        bmark_end(h);
    }
    if (mode == MODE_EVAL) return;
    const int M = h->mp.mem;
    if (M <= 4) blaunch_memory_mix<V, 4>(h, cur);
    else if (M <= 8) blaunch_memory_mix<V, 8>(h, cur);
    else if (M <= 16) blaunch_memory_mix<V, 16>(h, cur);
    else blaunch_memory_mix<V, 32>(h, cur);
}

int launches_per_iter(bh_t h, int64_t g) {
    const bool kkt = h->kkt_every > 0 && g >= 1 && (g - 1) % h->kkt_every == 0;
    const bool mix = h->mp.method != 0 && h->mp.mem > 0;
    return 4 + (kkt ? 1 : 0) + (mix ? 3 : 0);
}

template <typename V> bool blaunch_chunk_graph(bh_t h, int64_t g0) {
    if (!h->use_graphs || h->prof_on) return false;
    const int64_t phase = h->kkt_every > 0 ? (g0 - 1) % h->kkt_every : 0;
    const int parity = (int)(g0 & 1);
    const double tol = h->mp.tol;
    int64_t nl = 0;
    for (int64_t c = 0; c < B_CHUNK_ITERS; ++c) nl += launches_per_iter(h, g0 + c);
    for (auto &e : h->graphs)
        if (e.phase == phase && e.parity == parity && e.kkt_every == h->kkt_every && e.tol == tol) {
            if (cudaGraphLaunch(e.exec, h->stream) != cudaSuccess) { cudaGetLastError(); return false; }
            h->launches += nl;
            return true;
        }
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        h->use_graphs = false;
        return false;
    }
    if (h->graphs.size() >= 8) bdrop_graphs(h);
    cudaStream_t user = h->stream;
    h->stream = h->cap_stream;
    cudaGraph_t graph = nullptr;
    bool ok = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    const int64_t saved = h->launches;
    if (ok) {
        for (int64_t c = 0; c < B_CHUNK_ITERS; ++c) blaunch_iteration<V>(h, g0 + c, MODE_ITER);
        ok = cudaStreamEndCapture(h->cap_stream, &graph) == cudaSuccess;
    }
    h->stream = user;
    h->launches = saved;
    cudaGraphExec_t exec = nullptr;
    if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        h->use_graphs = false;
        return false;
    }
    h->graphs.push_back({exec, phase, parity, h->kkt_every, tol});
    if (cudaGraphLaunch(exec, h->stream) != cudaSuccess) { cudaGetLastError(); return false; }
    h->launches += nl;
    return true;
}

// Per-problem headers into hdr_host (one strided copy) after a stream sync.
aapdhg_status bread_headers(bh_t h) {
    BCK(h, cudaMemcpy2DAsync(h->hdr_host, HDR, h->stb, sizeof(DevState), HDR, h->nprob,
                             cudaMemcpyDeviceToHost, h->stream));
    BCK(h, cudaStreamSynchronize(h->stream));
    bcollect(h);
    return AAPDHG_OK;
}

const DevState *hdr(bh_t h, int32_t p) { return reinterpret_cast<const DevState *>(h->hdr_host + HDR * p); }

// Start of a solve call: rings, autotuning, then u^1 = T u^0 of every problem
// (first call) or a re-test of converged problems (later calls).  Enqueues
// work only.
template <typename V> aapdhg_status bbegin(bh_t h, double tol, int32_t kkt_every) {
    h->mp.tol = tol;
    h->kkt_every = kkt_every;
    aapdhg_status s = AAPDHG_OK;
    if (h->mp.method != 0 && h->mp.mem > 0 && (s = bensure_rings<V>(h)) != AAPDHG_OK) return s;
    if (h->autotune && !h->tuned && (s = bautotune<V>(h)) != AAPDHG_OK) return s;
    if (h->g == 0) {
        if (h->pw_period > 0) {                  // snapshot u^0 for the first update
            k_pw_delta_b<V><<<bview<V>(h).nchunk, BLOCK, 0, h->stream>>>(
                bprob<V>(h).UP, (V *)h->pw_snap, bview<V>(h), 0, 1, h->pw_part);
            h->launches += 1;
        }
        blaunch_iteration<V>(h, 0, MODE_ITER);   // u^1 = T u^0 and g^0 of every problem
        h->g = 1;
    } else {
        k_batch_clear_done<<<(h->nprob + 255) / 256, 256, 0, h->stream>>>(h->stb, h->nprob);
        h->launches += 1;
    }
    BCK(h, cudaGetLastError());
    return AAPDHG_OK;
}

// Primal weight update of every running problem at its iterate u^k, k = h->g
// (the iteration about to be launched works on u^g): enqueued only.
template <typename V> aapdhg_status bpw_update(bh_t h) {
    Prob<V> &P = bprob<V>(h);
    BatchView<V> &B = bview<V>(h);
    const int cur = (int)(h->g & 1);
    k_pw_delta_b<V><<<B.nchunk, BLOCK, 0, h->stream>>>(P.UP, (V *)h->pw_snap, B, cur, 0, h->pw_part);
    k_pw_apply_b<V><<<(h->nprob + 127) / 128, 128, 0, h->stream>>>(B, h->pw_part, h->pw_w, h->pw_alpha,
                                                                    h->pw_upd, h->pw);
    h->launches += 2;
    if (h->pw_dhat) {
        k_dhat_blend_b<V><<<B.nchunk, BLOCK, 0, h->stream>>>(const_cast<V *>(P.dh), (const V *)h->pw_dh_base, B,
                                                              h->pw_w, h->pw_alpha, h->pw_upd);
        h->launches += 1;
    }
    BCK(h, cudaGetLastError());
    return AAPDHG_OK;
}

// Enqueue n batch iterations (CUDA graphs for full chunks); with the primal
// weight update on, the run is cut at the update points k = 0 mod U_P, each
// update enqueued before its iteration.
template <typename V> aapdhg_status blaunch_chunk(bh_t h, int64_t n) {
    while (n > 0) {
        int64_t c = n;
        if (h->pw_period > 0) {
            const int64_t r = h->g % h->pw_period;
            if (r == 0 && h->pw_last_g != h->g) {
                aapdhg_status s = bpw_update<V>(h);
                if (s != AAPDHG_OK) return s;
                h->pw_last_g = h->g;
            }
            c = std::min<int64_t>(c, h->pw_period - r);
        }
        if (!(c == B_CHUNK_ITERS && blaunch_chunk_graph<V>(h, h->g)))
            for (int64_t i = 0; i < c; ++i) blaunch_iteration<V>(h, h->g + i, MODE_ITER);
        BCK(h, cudaGetLastError());
        h->g += c;
        n -= c;
    }
    return AAPDHG_OK;
}

bool ball_stopped(bh_t h) {
    for (int32_t p = 0; p < h->nprob; ++p)
        if (!hdr(h, p)->done && !hdr(h, p)->error) return false;
    return true;
}

aapdhg_status bfinal_status(bh_t h) {
    bool any_err = false, all_done = true;
    for (int32_t p = 0; p < h->nprob; ++p) {
        any_err |= hdr(h, p)->error != 0;
        all_done &= hdr(h, p)->done != 0;
    }
    if (any_err) {
        h->err = "NaN or Inf in the iterate of at least one problem (see aapdhg_batch_get_status)";
        return AAPDHG_ERR_NUMERIC;
    }
    return all_done ? AAPDHG_OK : AAPDHG_NOT_CONVERGED;
}

template <typename V> aapdhg_status biterate(bh_t h, int64_t max_iters, double tol, int32_t kkt_every,
                                            int64_t *iters_done) {
    aapdhg_status s = bbegin<V>(h, tol, kkt_every);
    if (s != AAPDHG_OK) return s;
    if ((s = bread_headers(h)) != AAPDHG_OK) return s;
    int64_t launched = 0;
    bool stop = ball_stopped(h);
    while (launched < max_iters && !stop) {
        const int64_t chunk = std::min<int64_t>(B_CHUNK_ITERS, max_iters - launched);
        if ((s = blaunch_chunk<V>(h, chunk)) != AAPDHG_OK) return s;
        launched += chunk;
        if ((s = bread_headers(h)) != AAPDHG_OK) return s;
        stop = ball_stopped(h);
    }
    if (iters_done) *iters_done = launched;
    return bfinal_status(h);
}

template <typename V> aapdhg_status bget_iterate(bh_t h, double *x, double *y) {
    typedef typename Vec2<V>::T V2;
    Prob<V> &P = bprob<V>(h);
    const int cur = (int)(h->g & 1);
    std::vector<V2> up(h->N);
    BCK(h, cudaMemcpyAsync(up.data(), P.UP, sizeof(V2) * h->N, cudaMemcpyDeviceToHost, h->stream));
    BCK(h, cudaStreamSynchronize(h->stream));
    for (int32_t p = 0; p < h->nprob; ++p) {
        const int32_t *px = h->perm_x.data() + h->xcat[p];
        const int32_t *py = h->perm_y.data() + h->ycat[p];
        if (x)
            for (int32_t j = 0; j < h->n[p]; ++j) {
                const int64_t e = h->xoff[p] + j;
                const double v = (double)(cur ? up[e].y : up[e].x);
                x[h->xcat[p] + px[j]] = h->scaled ? v * h->dc[e] : v;
            }
        if (y)
            for (int32_t i = 0; i < h->m[p]; ++i) {
                const int64_t r = h->yoff[p] + i;
                const double v = (double)(cur ? up[h->n_tot + r].y : up[h->n_tot + r].x);
                y[h->ycat[p] + py[i]] = h->scaled ? v * h->dr[r] : v;
            }
    }
    return AAPDHG_OK;
}

// One member's current iterate (caller order) and the KKT values of its last
// test, read from its own ranges only.
template <typename V> aapdhg_status bget_member(bh_t h, int32_t p, double *x, double *y, double *kkt6,
                                                int64_t *st6) {
    typedef typename Vec2<V>::T V2;
    Prob<V> &P = bprob<V>(h);
    const int cur = (int)(h->g & 1);
    std::vector<V2> ux(h->n[p]), uy(std::max(h->m[p], 1));
    DevState d;
    BCK(h, cudaMemcpyAsync(ux.data(), P.UP + h->xoff[p], sizeof(V2) * h->n[p], cudaMemcpyDeviceToHost,
                           h->stream));
    if (h->m[p] > 0)
        BCK(h, cudaMemcpyAsync(uy.data(), P.UP + h->n_tot + h->yoff[p], sizeof(V2) * h->m[p],
                               cudaMemcpyDeviceToHost, h->stream));
    BCK(h, cudaMemcpyAsync(&d, h->stb + p, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
    BCK(h, cudaStreamSynchronize(h->stream));
    const int32_t *px = h->perm_x.data() + h->xcat[p];
    const int32_t *py = h->perm_y.data() + h->ycat[p];
    if (x)
        for (int32_t j = 0; j < h->n[p]; ++j) {
            const double v = (double)(cur ? ux[j].y : ux[j].x);
            x[px[j]] = h->scaled ? v * h->dc[h->xoff[p] + j] : v;
        }
    if (y)
        for (int32_t i = 0; i < h->m[p]; ++i) {
            const double v = (double)(cur ? uy[i].y : uy[i].x);
            y[py[i]] = h->scaled ? v * h->dr[h->yoff[p] + i] : v;
        }
    if (kkt6)
        for (int k = 0; k < 6; ++k) kkt6[k] = d.kkt[k];
    if (st6) {
        st6[0] = d.it;
        st6[1] = d.n_aa;
        st6[2] = d.n_pd;
        st6[3] = d.n_lsfail;
        st6[4] = d.done != 0;
        st6[5] = d.error != 0;
    }
    return AAPDHG_OK;
}

template <typename V> aapdhg_status bget_kkt(bh_t h, double *out) {
    blaunch_iteration<V>(h, h->g, MODE_EVAL);
    BCK(h, cudaGetLastError());
    BCK(h, cudaMemcpy2DAsync(out, 6 * sizeof(double), reinterpret_cast<const char *>(h->stb) + offsetof(DevState, kkt),
                             sizeof(DevState), 6 * sizeof(double), h->nprob, cudaMemcpyDeviceToHost, h->stream));
    BCK(h, cudaStreamSynchronize(h->stream));
    bcollect(h);
    return AAPDHG_OK;
}

// Power iteration on every K_p' K_p at once (the Sec. 5.1 step-size rule): the
// packed SpMVs, then per-problem norms and normalisation over each problem's
// variable segment.  Each problem's start vector is the single-LP one for the
// same seed (splitmix64 over its internal variable order).
template <typename V> aapdhg_status bestimate_norms(bh_t h, int32_t iters, uint64_t seed, double *norms) {
    Prob<V> &P = bprob<V>(h);
    const size_t mark = h->allocs.size();
    V *v = (V *)bdev_alloc(h, sizeof(V) * h->n_tot);
    V *w = (V *)bdev_alloc(h, sizeof(V) * std::max<int64_t>(h->m_tot, 1));
    double *part = (double *)bdev_alloc(h, sizeof(double) * std::max(P.grid1, P.grid2));
    double *ss = (double *)bdev_alloc(h, sizeof(double) * h->nprob);
    int64_t *off = (int64_t *)bdev_alloc(h, sizeof(int64_t) * (h->nprob + 1));
    if (!v || !w || !part || !ss || !off) return bfail(h, AAPDHG_ERR_OOM, "power iteration buffers");
    std::vector<V> hv(h->n_tot, V(0));
    std::vector<int64_t> hoff(h->nprob + 1);
    for (int32_t p = 0; p < h->nprob; ++p) {
        uint64_t z = seed ? seed : 0x9E3779B97F4A7C15ull;
        for (int32_t j = 0; j < h->n[p]; ++j) {
            z += 0x9E3779B97F4A7C15ull;
            uint64_t t = z;
            t = (t ^ (t >> 30)) * 0xBF58476D1CE4E5B9ull;
            t = (t ^ (t >> 27)) * 0x94D049BB133111EBull;
            t ^= t >> 31;
            hv[h->xoff[p] + j] = (V)((double)(t >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0);
        }
        hoff[p] = h->xoff[p];
    }
    hoff[h->nprob] = h->n_tot;
    BCK(h, cudaMemcpyAsync(v, hv.data(), sizeof(V) * h->n_tot, cudaMemcpyHostToDevice, h->stream));
    BCK(h, cudaMemcpyAsync(off, hoff.data(), sizeof(int64_t) * (h->nprob + 1), cudaMemcpyHostToDevice, h->stream));
    for (int32_t t = 0; t < iters; ++t) {
        if (h->m_tot > 0) k_spmv_plain<V, false><<<P.grid2, BLOCK, 0, h->stream>>>(P.K, v, w, part);
        k_spmv_plain<V, false><<<P.grid1, BLOCK, 0, h->stream>>>(P.KT, w, v, part);
        k_seg_sumsq<V><<<h->nprob, BLOCK, 0, h->stream>>>(v, off, ss);
        k_seg_scale<V><<<h->nprob, BLOCK, 0, h->stream>>>(v, off, ss);
        BCK(h, cudaGetLastError());
    }
    std::vector<double> hs(h->nprob);
    BCK(h, cudaMemcpyAsync(hs.data(), ss, sizeof(double) * h->nprob, cudaMemcpyDeviceToHost, h->stream));
    BCK(h, cudaStreamSynchronize(h->stream));
    // ||K'K v|| of the last (unit) v is sqrt(ss); the norm of K is its square root
    for (int32_t p = 0; p < h->nprob; ++p) norms[p] = sqrt(sqrt(hs[p]));
    while (h->allocs.size() > mark) {
        auto a = h->allocs.back();
        h->allocs.pop_back();
        h->bytes -= (int64_t)a.bytes;
        raw_free(a.p);
    }
    return AAPDHG_OK;
}

template <typename V> aapdhg_status bset_scaling(bh_t h, int32_t ruiz_iters, int32_t pc) {
    Prob<V> &P = bprob<V>(h);
    const int64_t m = h->m_tot, n = h->n_tot;
    V *dr = (V *)bdev_alloc(h, sizeof(V) * std::max<int64_t>(m, 1));
    V *dc = (V *)bdev_alloc(h, sizeof(V) * n);
    V *tr = (V *)bdev_alloc(h, sizeof(V) * std::max<int64_t>(m, 1));
    V *tc = (V *)bdev_alloc(h, sizeof(V) * n);
    V *scx = (V *)bdev_alloc(h, sizeof(V) * n);
    V *scy = (V *)bdev_alloc(h, sizeof(V) * std::max<int64_t>(m, 1));
    if (!dr || !dc || !tr || !tc || !scx || !scy) return bfail(h, AAPDHG_ERR_OOM, "scaling buffers");
    cudaStream_t s = h->stream;
    const int gv = bgrid(h, (h->N + BLOCK - 1) / BLOCK, 4);
    const int gr = bgrid(h, (h->N + WARPS - 1) / WARPS, 8);
    k_fill<V><<<gv, BLOCK, 0, s>>>(dr, V(1), m);
    k_fill<V><<<gv, BLOCK, 0, s>>>(dc, V(1), n);
    for (int32_t pass = 0; pass < ruiz_iters + (pc ? 1 : 0); ++pass) {
        const int sum = pass >= ruiz_iters;
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
    k_vdiv<V><<<gv, BLOCK, 0, s>>>(const_cast<V *>(P.lo), dc, n);
    k_vdiv<V><<<gv, BLOCK, 0, s>>>(const_cast<V *>(P.hi), dc, n);
    k_vinv<V><<<gv, BLOCK, 0, s>>>(scx, dc, n);
    k_vinv<V><<<gv, BLOCK, 0, s>>>(scy, dr, m);
    BCK(h, cudaGetLastError());
    std::vector<V> hr(std::max<int64_t>(m, 1)), hc(n);
    BCK(h, cudaMemcpyAsync(hr.data(), dr, sizeof(V) * m, cudaMemcpyDeviceToHost, s));
    BCK(h, cudaMemcpyAsync(hc.data(), dc, sizeof(V) * n, cudaMemcpyDeviceToHost, s));
    BCK(h, cudaStreamSynchronize(s));
    h->dr.assign(hr.begin(), hr.begin() + m);
    h->dc.assign(hc.begin(), hc.end());
    P.sc_x = scx;
    P.sc_y = m > 0 ? scy : nullptr;
    k_dhat<V><<<gr, BLOCK, 0, s>>>(P.KT, P.K, P.n, P.m, h->dhat_mode < 0 ? 1 : h->dhat_mode,
                                   const_cast<V *>(P.dh));
    BCK(h, cudaGetLastError());
    h->pw_base_valid = false;
    h->scaled = true;
    return AAPDHG_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

aapdhg_status aapdhg_batch_create(int32_t nprob, const int32_t *m, const int32_t *n, const int64_t *nnz,
                                  const int64_t *row_ptr, const int32_t *col_idx, const double *val,
                                  const int8_t *row_sense, const double *q, const double *c,
                                  const double *lb, const double *ub, int32_t precision,
                                  void *cuda_stream, aapdhg_batch_t *out) {
    NvtxRange range("aapdhg_batch_create");
    if (!out) return bfail(nullptr, AAPDHG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (nprob < 1 || nprob >= (1 << 25) || !m || !n || !nnz || !row_ptr)
        return bfail(nullptr, AAPDHG_ERR_INVALID, "need 1 <= nprob < 2^25 and non-NULL size arrays");
    if (precision != AAPDHG_FP64 && precision != AAPDHG_MIXED)
        return bfail(nullptr, AAPDHG_ERR_INVALID, "unknown precision");
    // offsets of each problem in the concatenated caller arrays; validation
    std::vector<int64_t> rpc(nprob), kc(nprob), xc(nprob), yc(nprob);
    int64_t R = 0, Z = 0, X = 0, Y = 0, xt = 0, yt = 0;
    for (int32_t p = 0; p < nprob; ++p) {
        if (m[p] < 0 || n[p] < 1 || nnz[p] < 0)
            return bfail(nullptr, AAPDHG_ERR_INVALID, "problem " + std::to_string(p) + ": need m >= 0, n >= 1, nnz >= 0");
        rpc[p] = R; kc[p] = Z; xc[p] = X; yc[p] = Y;
        R += m[p] + 1; Z += nnz[p]; X += n[p]; Y += m[p];
        xt += (n[p] + 3) & ~3; yt += (m[p] + 3) & ~3;
    }
    if (Z >= ((int64_t)1 << 31) || xt + yt >= ((int64_t)1 << 31))
        return bfail(nullptr, AAPDHG_ERR_INVALID, "the packed batch needs < 2^31 nonzeros and elements");
    // problems checked in parallel (weighted by nonzeros); the lowest failing one is reported
    std::vector<int64_t> zpre(nprob + 1, 0);
    for (int32_t p = 0; p < nprob; ++p) zpre[p + 1] = zpre[p] + nnz[p] + m[p] + n[p];
    const std::vector<int64_t> pcuts = weight_cuts(zpre.data(), nprob, host_threads(zpre[nprob]));
    std::vector<int32_t> bad_p(pcuts.size() - 1, nprob);
    std::vector<std::string> bad_why(pcuts.size() - 1);
    run_ranges(pcuts, [&](int t, int64_t lo, int64_t hi) {
        for (int64_t p = lo; p < hi; ++p) {
            std::string why = validate_lp(
                m[p], n[p], nnz[p], row_ptr + rpc[p], nnz[p] ? col_idx + kc[p] : nullptr,
                nnz[p] ? val + kc[p] : nullptr, m[p] ? row_sense + yc[p] : nullptr, m[p] ? q + yc[p] : nullptr,
                c ? c + xc[p] : nullptr, lb ? lb + xc[p] : nullptr, ub ? ub + xc[p] : nullptr);
            if (!why.empty()) {
                bad_p[t] = (int32_t)p;
                bad_why[t] = std::move(why);
                return;
            }
        }
    });
    {
        size_t tb = 0;
        for (size_t t = 1; t < bad_p.size(); ++t)
            if (bad_p[t] < bad_p[tb]) tb = t;
        if (bad_p[tb] < nprob)
            return bfail(nullptr, AAPDHG_ERR_INVALID, "problem " + std::to_string(bad_p[tb]) + ": " + bad_why[tb]);
    }

    bh_t h = new (std::nothrow) aapdhg_batch_s();
    if (!h) return bfail(nullptr, AAPDHG_ERR_OOM, "host allocation");
    h->nprob = nprob;
    h->prec = precision;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) {
        if (cuda_stream) h->stream = (cudaStream_t)cuda_stream;
        else { e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking); h->own_stream = true; }
    }
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->hdr_host, HDR * (size_t)nprob);
    if (e != cudaSuccess) {
        std::string msg = std::string("CUDA setup: ") + cudaGetErrorString(e);
        if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
        delete h;
        return bfail(nullptr, AAPDHG_ERR_CUDA, msg);
    }
    h->m.assign(m, m + nprob);
    h->n.assign(n, n + nprob);
    h->nxp.resize(nprob);
    h->nyp.resize(nprob);
    h->xoff.resize(nprob);
    h->yoff.resize(nprob);
    h->xcat = xc;
    h->ycat = yc;
    for (int32_t p = 0; p < nprob; ++p) {
        h->nxp[p] = (n[p] + 3) & ~3;
        h->nyp[p] = (m[p] + 3) & ~3;
        h->xoff[p] = h->n_tot;
        h->yoff[p] = h->m_tot;
        h->n_tot += h->nxp[p];
        h->m_tot += h->nyp[p];
    }
    h->N = h->n_tot + h->m_tot;
    h->Npad = (h->N + 63) & ~(int64_t)63;
    h->lo_x.assign(lb, lb + X);
    h->hi_x.assign(ub, ub + X);
    h->sense.assign(row_sense ? row_sense : (const int8_t *)nullptr, row_sense ? row_sense + Y : nullptr);
    h->tau.assign(nprob, 0.0);
    h->sigma.assign(nprob, 0.0);

    // per-problem renumbering, packed into one K and one K': problem p's
    // nonzeros occupy [kc[p], kc[p] + nnz[p]) of both, so the problems are
    // renumbered in parallel (weighted by nonzeros) and written in place
    HostCSR K, KT;
    K.rows = (int32_t)h->m_tot;
    KT.rows = (int32_t)h->n_tot;
    K.rp.assign(h->m_tot + 1, 0);
    KT.rp.assign(h->n_tot + 1, 0);
    K.ci.resize(Z); K.val.resize(Z); KT.ci.resize(Z); KT.val.resize(Z);
    std::vector<double> cv(h->n_tot, 0.0), qv(std::max<int64_t>(h->m_tot, 1), 0.0);
    std::vector<double> lov(h->N, 0.0), hiv(h->N, 0.0), pnorm(2 * (size_t)nprob);
    std::vector<RowSeg> segK, segKT;
    for (int32_t p = 0; p < nprob; ++p) {
        segK.push_back(RowSeg{(int32_t)h->yoff[p], h->nyp[p], p});
        segKT.push_back(RowSeg{(int32_t)h->xoff[p], h->nxp[p], p});
    }
    h->perm_x.resize(X);
    h->perm_y.resize(Y);
    run_ranges(pcuts, [&](int, int64_t lo, int64_t hi) {
        for (int64_t p = lo; p < hi; ++p) {
            std::vector<int32_t> px, py;
            HostCSR Kp, KTp;
            const int32_t mp_ = m[p], np_ = n[p];
            build_internal(mp_, np_, row_ptr + rpc[p], nnz[p] ? col_idx + kc[p] : nullptr,
                           nnz[p] ? val + kc[p] : nullptr, px, py, Kp, KTp);
            const int64_t xo = h->xoff[p], yo = h->yoff[p], z0 = kc[p];
            for (int32_t ii = 0; ii < h->nyp[p]; ++ii)
                K.rp[yo + ii + 1] = (int32_t)(z0 + (ii < mp_ ? Kp.rp[ii + 1] : nnz[p]));
            for (int64_t k = 0; k < nnz[p]; ++k) {
                K.ci[z0 + k] = (int32_t)(xo + Kp.ci[k]);
                K.val[z0 + k] = Kp.val[k];
            }
            for (int32_t jj = 0; jj < h->nxp[p]; ++jj)
                KT.rp[xo + jj + 1] = (int32_t)(z0 + (jj < np_ ? KTp.rp[jj + 1] : nnz[p]));
            for (int64_t k = 0; k < nnz[p]; ++k) {
                KT.ci[z0 + k] = (int32_t)(yo + KTp.ci[k]);
                KT.val[z0 + k] = KTp.val[k];
            }
            double q2 = 0.0, c2 = 0.0;
            for (int32_t j = 0; j < np_; ++j) {
                const int64_t oj = xc[p] + px[j];
                cv[xo + j] = c[oj];
                lov[xo + j] = lb[oj];
                hiv[xo + j] = ub[oj];
                c2 += c[oj] * c[oj];
            }
            for (int32_t i = 0; i < h->nyp[p]; ++i) {
                const int64_t e2 = h->n_tot + yo + i;
                hiv[e2] = INFINITY;
                lov[e2] = -INFINITY;
                if (i < mp_) {
                    const int64_t oi = yc[p] + py[i];
                    qv[yo + i] = q[oi];
                    lov[e2] = row_sense[oi] == AAPDHG_ROW_GE ? 0.0 : -INFINITY;
                    q2 += q[oi] * q[oi];
                }
            }
            pnorm[2 * p] = sqrt(q2);
            pnorm[2 * p + 1] = sqrt(c2);
            std::copy(px.begin(), px.end(), h->perm_x.begin() + xc[p]);
            std::copy(py.begin(), py.end(), h->perm_y.begin() + yc[p]);
        }
    });
    qv.resize(std::max<int64_t>(h->m_tot, 1));
    aapdhg_status s = precision == AAPDHG_FP64
                          ? bsetup<double>(h, K, KT, segK, segKT, cv, qv, lov, hiv, pnorm)
                          : bsetup<float>(h, K, KT, segK, segKT, cv, qv, lov, hiv, pnorm);
    if (s == AAPDHG_OK) {
        h->mp.method = AAPDHG_AA; h->mp.mem = 5; h->mp.D = 10.0; h->mp.eps = 1.0;
        h->mp.eta = 1e-10; h->mp.beta = 1.0; h->mp.c_s = 0.2; h->mp.kappa = 1e8; h->mp.c_div = 1.0;
        h->mp.faa_adaptive = 1;
        aapdhg_batch_set_start(h, nullptr, nullptr);
        s = h->sticky;
    }
    if (s != AAPDHG_OK) {
        g_batch_create_err = h->err;
        aapdhg_batch_destroy(h);
        return s;
    }
    *out = h;
    return AAPDHG_OK;
}

aapdhg_status aapdhg_batch_set_steps(aapdhg_batch_t h, const double *tau, const double *sigma) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (!tau || !sigma) return bfail(h, AAPDHG_ERR_INVALID, "tau and sigma arrays are required");
    for (int32_t p = 0; p < h->nprob; ++p)
        if (!(tau[p] > 0) || !(sigma[p] > 0) || !std::isfinite(tau[p]) || !std::isfinite(sigma[p]))
            return bfail(h, AAPDHG_ERR_INVALID, "tau and sigma must be finite and > 0");
    h->tau.assign(tau, tau + h->nprob);
    h->sigma.assign(sigma, sigma + h->nprob);
    aapdhg_status s = bupload_steps(h);
    if (s != AAPDHG_OK) return s;
    bdrop_graphs(h);
    return breset_any(h);
}

aapdhg_status aapdhg_batch_estimate_norms(aapdhg_batch_t h, int32_t iters, uint64_t seed, double *norms) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (!norms || iters < 1) return bfail(h, AAPDHG_ERR_INVALID, "bad arguments");
    return h->prec == AAPDHG_FP64 ? bestimate_norms<double>(h, iters, seed, norms)
                                  : bestimate_norms<float>(h, iters, seed, norms);
}

aapdhg_status aapdhg_batch_set_method(aapdhg_batch_t h, int32_t method, int32_t m_A, double D, double eps,
                                      double eta, double beta, double c_s, double kappa, double c_div,
                                      int32_t dhat_mode, int32_t faa_adaptive) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (method < 0 || method > 2 || m_A < 0 || m_A > AAPDHG_MAX_MEMORY || !(D > 0) || !(eps > 0) ||
        !(eta >= 0) || !(beta > 0 && beta <= 1) || !(c_s > 0 && c_s <= 1) || !(kappa > 0) ||
        !(c_div >= 1) || (dhat_mode != 0 && dhat_mode != 1))
        return bfail(h, AAPDHG_ERR_INVALID, "method parameters out of range");
    h->mp.method = method; h->mp.mem = m_A; h->mp.D = D; h->mp.eps = eps; h->mp.eta = eta;
    h->mp.beta = beta; h->mp.c_s = c_s; h->mp.kappa = kappa; h->mp.c_div = c_div;
    h->mp.faa_adaptive = faa_adaptive ? 1 : 0;
    bdrop_graphs(h);
    if (dhat_mode != h->dhat_mode) {
        const int gD = bgrid(h, (h->N + WARPS - 1) / WARPS, 8);
        if (h->prec == AAPDHG_FP64)
            k_dhat<double><<<gD, BLOCK, 0, h->stream>>>(h->pd.KT, h->pd.K, h->pd.n, h->pd.m, dhat_mode,
                                                        const_cast<double *>(h->pd.dh));
        else
            k_dhat<float><<<gD, BLOCK, 0, h->stream>>>(h->pf.KT, h->pf.K, h->pf.n, h->pf.m, dhat_mode,
                                                       const_cast<float *>(h->pf.dh));
        BCK(h, cudaGetLastError());
        h->dhat_mode = dhat_mode;
        h->pw_base_valid = false;
    }
    return breset_any(h);
}

aapdhg_status aapdhg_batch_set_scaling(aapdhg_batch_t h, int32_t ruiz_iters, int32_t pock_chambolle) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (h->scaled || ruiz_iters < 0 || ruiz_iters > 1000)
        return bfail(h, AAPDHG_ERR_INVALID, "scaling is applied at most once, with 0..1000 Ruiz passes");
    bdrop_graphs(h);
    aapdhg_status s = h->prec == AAPDHG_FP64 ? bset_scaling<double>(h, ruiz_iters, pock_chambolle)
                                             : bset_scaling<float>(h, ruiz_iters, pock_chambolle);
    if (s != AAPDHG_OK) return s;
    return breset_any(h);
}

aapdhg_status aapdhg_batch_set_primal_weight(aapdhg_batch_t h, int64_t period, double theta, double eps_zero,
                                             int32_t dhat_blend, double rho_min, double alpha_dec,
                                             double alpha_inc) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (period < 0 || !(theta >= 0 && theta <= 1) || !(eps_zero >= 0) || !std::isfinite(rho_min) ||
        !(alpha_dec >= 0 && alpha_dec <= 1) || !(alpha_inc >= 0 && alpha_inc <= 1))
        return bfail(h, AAPDHG_ERR_INVALID, "primal weight parameters out of range");
    const size_t sv = h->prec == AAPDHG_FP64 ? 8 : 4;
    if (period > 0) {
        const int32_t nchunk = h->prec == AAPDHG_FP64 ? h->bd.nchunk : h->bf.nchunk;
        if (!h->pw_snap) h->pw_snap = bdev_alloc(h, sv * h->N);
        if (!h->pw_dh_base) {
            h->pw_dh_base = bdev_alloc(h, sv * h->N);
            h->pw_base_valid = false;
        }
        if (!h->pw_part) h->pw_part = (double *)bdev_alloc(h, sizeof(double) * std::max(nchunk, 1));
        if (!h->pw_w) h->pw_w = (double *)bdev_alloc(h, sizeof(double) * 3 * h->nprob);
        if (!h->pw_alpha) h->pw_alpha = (double *)bdev_alloc(h, sizeof(double) * h->nprob);
        if (!h->pw_upd) h->pw_upd = (int32_t *)bdev_alloc(h, sizeof(int32_t) * h->nprob);
        if (!h->pw_snap || !h->pw_dh_base || !h->pw_part || !h->pw_w || !h->pw_alpha || !h->pw_upd)
            return bfail(h, AAPDHG_ERR_OOM, "primal weight buffers");
    } else if (h->pw_period > 0) {
        // back to fixed steps: the given steps and the base D-hat
        aapdhg_status s = bupload_steps(h);
        if (s != AAPDHG_OK) return s;
        if (h->pw_base_valid)
            BCK(h, cudaMemcpyAsync(h->prec == AAPDHG_FP64 ? (void *)h->pd.dh : (void *)h->pf.dh, h->pw_dh_base,
                                   sv * (size_t)h->N, cudaMemcpyDeviceToDevice, h->stream));
    }
    h->pw_period = period;
    h->pw = PwParams{theta, eps_zero, rho_min, alpha_dec, alpha_inc};
    h->pw_dhat = dhat_blend ? 1 : 0;
    h->bf.pw_on = h->bd.pw_on = period > 0 ? 1 : 0;
    bdrop_graphs(h);
    return breset_any(h);
}

aapdhg_status aapdhg_batch_set_start(aapdhg_batch_t h, const double *x0, const double *y0) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    const size_t X = h->lo_x.size(), Y = h->sense.size();
    h->x0.assign(X, 0.0);
    h->y0.assign(Y, 0.0);
    for (size_t j = 0; j < X; ++j) {
        const double v = x0 ? x0[j] : 0.0;
        if (!std::isfinite(v)) return bfail(h, AAPDHG_ERR_INVALID, "non-finite start");
        h->x0[j] = std::min(std::max(v, h->lo_x[j]), h->hi_x[j]);
    }
    for (size_t i = 0; i < Y; ++i) {
        double v = y0 ? y0[i] : 0.0;
        if (!std::isfinite(v)) return bfail(h, AAPDHG_ERR_INVALID, "non-finite start");
        if (h->sense[i] == AAPDHG_ROW_GE && v < 0) v = 0;
        h->y0[i] = v;
    }
    return breset_any(h);
}

aapdhg_status aapdhg_batch_reset(aapdhg_batch_t h) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    return breset_any(h);
}

aapdhg_status aapdhg_batch_set_tolerances(aapdhg_batch_t h, const double *tol) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (!tol) {
        h->bd.ptol = h->bf.ptol = nullptr;
        bdrop_graphs(h);
        return AAPDHG_OK;
    }
    for (int32_t p = 0; p < h->nprob; ++p)
        if (!(tol[p] >= 0)) return bfail(h, AAPDHG_ERR_INVALID, "tolerances must be >= 0");
    if (!h->ptol_dev) {
        h->ptol_dev = (double *)bdev_alloc(h, sizeof(double) * h->nprob);
        if (!h->ptol_dev) return bfail(h, AAPDHG_ERR_OOM, "tolerance array");
    }
    BCK(h, cudaMemcpyAsync(h->ptol_dev, tol, sizeof(double) * h->nprob, cudaMemcpyHostToDevice, h->stream));
    BCK(h, cudaStreamSynchronize(h->stream));
    if (h->prec == AAPDHG_FP64) h->bd.ptol = h->ptol_dev;
    else h->bf.ptol = h->ptol_dev;
    bdrop_graphs(h);
    return AAPDHG_OK;
}

aapdhg_status aapdhg_batch_iterate(aapdhg_batch_t h, int64_t max_iters, double tol, int32_t kkt_every,
                                   int64_t *iters_done) {
    NvtxRange range("aapdhg_batch_iterate");
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (max_iters < 0 || kkt_every < 0 || !(tol >= 0))
        return bfail(h, AAPDHG_ERR_INVALID, "need max_iters >= 0, kkt_every >= 0, tol >= 0");
    for (int32_t p = 0; p < h->nprob; ++p)
        if (!(h->tau[p] > 0)) return bfail(h, AAPDHG_ERR_INVALID, "set_steps must be called before iterate");
    return h->prec == AAPDHG_FP64 ? biterate<double>(h, max_iters, tol, kkt_every, iters_done)
                                  : biterate<float>(h, max_iters, tol, kkt_every, iters_done);
}

aapdhg_status aapdhg_batch_launch(aapdhg_batch_t h, int64_t n_iters, double tol, int32_t kkt_every) {
    NvtxRange range("aapdhg_batch_launch");
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (n_iters < 0 || kkt_every < 0 || !(tol >= 0))
        return bfail(h, AAPDHG_ERR_INVALID, "need n_iters >= 0, kkt_every >= 0, tol >= 0");
    for (int32_t p = 0; p < h->nprob; ++p)
        if (!(h->tau[p] > 0)) return bfail(h, AAPDHG_ERR_INVALID, "set_steps must be called before launch");
    const bool fp64 = h->prec == AAPDHG_FP64;
    aapdhg_status s = AAPDHG_OK;
    if (h->g == 0) {
        s = fp64 ? bbegin<double>(h, tol, kkt_every) : bbegin<float>(h, tol, kkt_every);
    } else {
        h->mp.tol = tol;
        h->kkt_every = kkt_every;
    }
    for (int64_t done = 0; s == AAPDHG_OK && done < n_iters; done += B_CHUNK_ITERS) {
        const int64_t n = std::min<int64_t>(B_CHUNK_ITERS, n_iters - done);
        s = fp64 ? blaunch_chunk<double>(h, n) : blaunch_chunk<float>(h, n);
    }
    return s;
}

aapdhg_status aapdhg_batch_poll(aapdhg_batch_t h, int32_t *all_stopped) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    aapdhg_status s = bread_headers(h);
    if (s != AAPDHG_OK) return s;
    if (all_stopped) *all_stopped = ball_stopped(h) ? 1 : 0;
    return AAPDHG_OK;
}

aapdhg_status aapdhg_batch_get_iterate(aapdhg_batch_t h, double *x, double *y) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    return h->prec == AAPDHG_FP64 ? bget_iterate<double>(h, x, y) : bget_iterate<float>(h, x, y);
}

aapdhg_status aapdhg_batch_get_member(aapdhg_batch_t h, int32_t p, double *x, double *y,
                                      double *kkt6, int64_t *status6) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (p < 0 || p >= h->nprob) return bfail(h, AAPDHG_ERR_INVALID, "problem index out of range");
    return h->prec == AAPDHG_FP64 ? bget_member<double>(h, p, x, y, kkt6, status6)
                                  : bget_member<float>(h, p, x, y, kkt6, status6);
}

aapdhg_status aapdhg_batch_get_kkt(aapdhg_batch_t h, double *out6) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (!out6) return bfail(h, AAPDHG_ERR_INVALID, "out6 is NULL");
    return h->prec == AAPDHG_FP64 ? bget_kkt<double>(h, out6) : bget_kkt<float>(h, out6);
}

aapdhg_status aapdhg_batch_get_status(aapdhg_batch_t h, int64_t *out6) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (!out6) return bfail(h, AAPDHG_ERR_INVALID, "out6 is NULL");
    aapdhg_status s = bread_headers(h);
    if (s != AAPDHG_OK) return s;
    for (int32_t p = 0; p < h->nprob; ++p) {
        const DevState *d = hdr(h, p);
        out6[6 * p] = d->it;
        out6[6 * p + 1] = d->n_aa;
        out6[6 * p + 2] = d->n_pd;
        out6[6 * p + 3] = d->n_lsfail;
        out6[6 * p + 4] = d->done != 0;
        out6[6 * p + 5] = d->error != 0;
    }
    return AAPDHG_OK;
}

aapdhg_status aapdhg_batch_profile_kernels(aapdhg_batch_t h, int32_t enable) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    BCK(h, cudaStreamSynchronize(h->stream));
    bcollect(h);
    h->prof_on = enable != 0;
    for (int k = 0; k < BK_N; ++k) { h->prof_ms[k] = 0; h->prof_n[k] = 0; }
    h->launches = 0;
    return AAPDHG_OK;
}

aapdhg_status aapdhg_batch_get_kernel_profile(aapdhg_batch_t h, int32_t kind, int64_t *launches,
                                              double *total_ms) {
    if (!h || !launches || !total_ms) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    BCK(h, cudaStreamSynchronize(h->stream));
    bcollect(h);
    if (kind == -1) { *launches = h->launches; *total_ms = 0.0; return AAPDHG_OK; }
    if (kind < 0 || kind >= BK_N) return bfail(h, AAPDHG_ERR_INVALID, "unknown kernel kind");
    *launches = h->prof_n[kind];
    *total_ms = h->prof_ms[kind];
    return AAPDHG_OK;
}

aapdhg_status aapdhg_batch_autotune(aapdhg_batch_t h, int32_t *shape_x, int32_t *shape_y, double *avg_us) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    aapdhg_status s = h->prec == AAPDHG_FP64 ? bautotune<double>(h) : bautotune<float>(h);
    if (s != AAPDHG_OK) return s;
    if (shape_x) *shape_x = h->shape_x;
    if (shape_y) *shape_y = h->shape_y;
    if (avg_us) for (int k = 0; k < 2 * NSHAPE; ++k) avg_us[k] = h->tune_us[k];
    return AAPDHG_OK;
}

aapdhg_status aapdhg_batch_set_layout(aapdhg_batch_t h, const int32_t *layout4) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (!layout4) return bfail(h, AAPDHG_ERR_INVALID, "layout4 is NULL");
    LayoutParams prm[2];
    for (int w = 0; w < 2; ++w) {
        const int32_t sm = layout4[2 * w], lc = layout4[2 * w + 1];
        if (sm < 1 || sm > 1024 || lc < 32 || lc > (1 << 20) || lc % 32)
            return bfail(h, AAPDHG_ERR_INVALID,
                         "layout: 1 <= sell_max <= 1024, long_chunk a multiple of 32 in [32, 2^20]");
        prm[w].sell_max = sm;
        prm[w].long_chunk = lc;
    }
    return h->prec == AAPDHG_FP64 ? bset_layout_t<double>(h, prm) : bset_layout_t<float>(h, prm);
}

aapdhg_status aapdhg_batch_autotune_layout(aapdhg_batch_t h, int32_t *layout4, double *avg_us) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    NvtxRange range("aapdhg_batch_autotune_layout");
    aapdhg_status s = h->prec == AAPDHG_FP64 ? bautotune_layout_t<double>(h) : bautotune_layout_t<float>(h);
    if (s != AAPDHG_OK) return s;
    if (layout4) {
        layout4[0] = h->lay[0].sell_max;
        layout4[1] = h->lay[0].long_chunk;
        layout4[2] = h->lay[1].sell_max;
        layout4[3] = h->lay[1].long_chunk;
    }
    if (avg_us) for (int k = 0; k < 2 * kNumLayoutCand; ++k) avg_us[k] = h->lay_us[k];
    return AAPDHG_OK;
}

aapdhg_status aapdhg_batch_set_task_shape(aapdhg_batch_t h, int32_t shape_x, int32_t shape_y) {
    if (!h) return AAPDHG_ERR_INVALID;
    if (h->sticky) return h->sticky;
    if (shape_x == -1 && shape_y == -1) {
        h->autotune = true;
        h->tuned = false;
        return AAPDHG_OK;
    }
    if (shape_x < 0 || shape_x >= NSHAPE || shape_y < 0 || shape_y >= NSHAPE)
        return bfail(h, AAPDHG_ERR_INVALID, "task shapes are 0 .. AAPDHG_TASK_SHAPES - 1, or both -1");
    h->autotune = false;
    bset_shapes(h, shape_x, shape_y);
    bdrop_graphs(h);
    return AAPDHG_OK;
}

aapdhg_status aapdhg_batch_device_bytes(aapdhg_batch_t h, int64_t *bytes) {
    if (!h || !bytes) return AAPDHG_ERR_INVALID;
    *bytes = h->bytes;
    return AAPDHG_OK;
}

const char *aapdhg_batch_last_error(aapdhg_batch_t h) {
    if (!h) return g_batch_create_err.c_str();
    return h->err.c_str();
}

void aapdhg_batch_destroy(aapdhg_batch_t h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    bdrop_graphs(h);
    for (auto e : h->ev) cudaEventDestroy(e);
    for (auto &a : h->allocs) raw_free(a.p);
    h->allocs.clear();
    if (h->hdr_host) cudaFreeHost(h->hdr_host);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"
