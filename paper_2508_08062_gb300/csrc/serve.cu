// Served stream of LPs (aapdhg_server_*): continuous batching on one GPU.
//
// Requests (an LP and its tolerance) arrive at any time.  Each scheduling
// round (aapdhg_server_step):
//   1. enqueues one chunk of iterations on every running cohort (a batch
//      handle of aapdhg_batch_*, on its own CUDA stream), without waiting;
//   2. while those run, admits waiting requests: in arrival order, as many as
//      the free device memory budget and the cohort size limit allow, form a
//      new cohort (packing, Ruiz + Pock-Chambolle scaling, per-problem power
//      iteration for the step sizes, per-problem tolerances); requests with a
//      tolerance below the mixed-precision limit go to FP64 cohorts;
//   3. polls every cohort; a member is finished when its KKT residual met its
//      tolerance (its iterate then stays frozen on the device), failed, or
//      reached the iteration cap.  A member that converged or failed hands its
//      result back at once (read from its own ranges), while the rest of its
//      cohort runs on; a cohort whose members are all finished hands back the
//      capped ones and frees its memory.
// So requests that arrive while others are on the GPU start as soon as
// memory allows, and the work of all cohorts overlaps on the device (each
// cohort's kernels are on its own stream).  Every member's iterates, Anderson
// memory and step sizes stay on the device from admission to retirement.
#include <chrono>
#include <cmath>
#include <deque>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/aapdhg.h"
#include "host.h"

namespace {

thread_local std::string g_server_create_err;

struct Request {
    int32_t m = 0, n = 0;
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> val, q, c, lb, ub;
    std::vector<int8_t> sense;
    double tol = 1e-4;
    int32_t prec = AAPDHG_MIXED;
    int32_t state = AAPDHG_REQ_WAITING;
    double t_submit = 0, t_admit = -1, t_done = -1;
    int64_t iters = 0;
    std::vector<double> x, y;
    double kkt[6] = {0, 0, 0, 0, 0, 0};
    int64_t est_bytes = 0;
    bool collected = false;       // result already read back
};

struct Cohort {
    aapdhg_batch_t b = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<int64_t> ids;
    int32_t prec = AAPDHG_MIXED;
    int64_t iters = 0;            // batch iterations enqueued
    int64_t bytes = 0;
};

}  // namespace

struct aapdhg_server_s {
    int32_t method = AAPDHG_AA, mem = 10;
    int32_t max_cohorts = 4, max_cohort_size = 64;
    int64_t max_iters = 100000;
    int64_t budget = 0;           // device bytes all cohorts may hold together
    int32_t kkt_every = 64;
    double mixed_tol_limit = 1e-5;  // tolerances below this are solved in FP64
    // primal weight update of the cohorts admitted from now on (0: off)
    int64_t pw_period = 0;
    double pw_theta = 0.5, pw_eps = 1e-10, pw_rho_min = 0.1, pw_alpha_dec = 0.1, pw_alpha_inc = 0.9;
    int32_t pw_dhat = 1;
    std::vector<Request> reqs;
    std::deque<int64_t> waiting[2];
    std::vector<Cohort> cohorts;
    int64_t held = 0;             // device bytes of the running cohorts
    std::chrono::steady_clock::time_point t0;
    std::string err;
    aapdhg_status sticky = AAPDHG_OK;
};

namespace {

double now_s(const aapdhg_server_s *s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

aapdhg_status sfail(aapdhg_server_t s, aapdhg_status st, const std::string &msg) {
    if (s) {
        if (s->sticky == AAPDHG_OK) { s->sticky = st; s->err = msg; }
    } else {
        g_server_create_err = msg;
    }
    return st;
}

// Device bytes a request needs in a cohort: K and K' as CSR plus their
// chunk / SELL copies (values and int32 indices), the iterate pairs and the
// per-element vectors, the two Anderson rings (33 slots) and the scaling
// buffers, in the cohort's precision.
int64_t estimate_bytes(const aapdhg_server_s *s, const Request &r) {
    const int64_t sv = r.prec == AAPDHG_FP64 ? 8 : 4;
    const int64_t Z = (int64_t)r.ci.size(), N = (int64_t)r.n + r.m + 8;
    const int64_t pw = s->pw_period > 0 ? 2 * N * sv : 0;    // snapshot and base D-hat
    return 4 * Z * (4 + sv) + N * sv * (2 * 33 + 24) + pw + 8 * (int64_t)(r.m + r.n) + 4096;
}

// Build one cohort from the first waiting requests of one precision class.
aapdhg_status admit(aapdhg_server_t s, int cls) {
    std::deque<int64_t> &wq = s->waiting[cls];
    std::vector<int64_t> ids;
    int64_t bytes = 0;
    while (!wq.empty() && (int32_t)ids.size() < s->max_cohort_size) {
        const Request &r = s->reqs[wq.front()];
        if (s->held + bytes + r.est_bytes > s->budget) break;
        bytes += r.est_bytes;
        ids.push_back(wq.front());
        wq.pop_front();
    }
    if (ids.empty()) {
        // nothing fits: a request larger than the whole budget can never run
        if (!wq.empty() && s->cohorts.empty() && s->reqs[wq.front()].est_bytes > s->budget) {
            Request &r = s->reqs[wq.front()];
            r.state = AAPDHG_REQ_REJECTED;
            r.t_done = now_s(s);
            wq.pop_front();
        }
        return AAPDHG_OK;
    }
    Cohort co;
    co.ids = ids;
    co.prec = cls == 1 ? AAPDHG_FP64 : AAPDHG_MIXED;
    if (cudaStreamCreateWithFlags(&co.stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return sfail(s, AAPDHG_ERR_CUDA, "cohort stream");
    }
    const int32_t k = (int32_t)ids.size();
    std::vector<int32_t> m(k), n(k);
    std::vector<int64_t> nnz(k), rp;
    std::vector<int32_t> ci;
    std::vector<double> val, q, c, lb, ub, tol(k);
    std::vector<int8_t> sense;
    for (int32_t i = 0; i < k; ++i) {
        const Request &r = s->reqs[ids[i]];
        m[i] = r.m;
        n[i] = r.n;
        nnz[i] = (int64_t)r.ci.size();
        rp.insert(rp.end(), r.rp.begin(), r.rp.end());
        ci.insert(ci.end(), r.ci.begin(), r.ci.end());
        val.insert(val.end(), r.val.begin(), r.val.end());
        sense.insert(sense.end(), r.sense.begin(), r.sense.end());
        q.insert(q.end(), r.q.begin(), r.q.end());
        c.insert(c.end(), r.c.begin(), r.c.end());
        lb.insert(lb.end(), r.lb.begin(), r.lb.end());
        ub.insert(ub.end(), r.ub.begin(), r.ub.end());
        tol[i] = r.tol;
    }
    aapdhg_status st = aapdhg_batch_create(k, m.data(), n.data(), nnz.data(), rp.data(), ci.data(),
                                           val.data(), sense.data(), q.data(), c.data(), lb.data(),
                                           ub.data(), co.prec, co.stream, &co.b);
    std::vector<double> norms(k), steps(k);
    if (st == AAPDHG_OK) st = aapdhg_batch_set_scaling(co.b, 10, 1);
    if (st == AAPDHG_OK) st = aapdhg_batch_estimate_norms(co.b, 100, 1, norms.data());
    if (st == AAPDHG_OK) {
        for (int32_t i = 0; i < k; ++i) steps[i] = norms[i] > 0 ? 0.9 / norms[i] : 1.0;
        st = aapdhg_batch_set_steps(co.b, steps.data(), steps.data());
    }
    if (st == AAPDHG_OK)
        st = aapdhg_batch_set_method(co.b, s->method, s->mem, 10.0, 1.0, 1e-10, 1.0, 0.2, 1e8, 1.0, 1, 1);
    if (st == AAPDHG_OK && s->pw_period > 0)
        st = aapdhg_batch_set_primal_weight(co.b, s->pw_period, s->pw_theta, s->pw_eps, s->pw_dhat,
                                            s->pw_rho_min, s->pw_alpha_dec, s->pw_alpha_inc);
    if (st == AAPDHG_OK) st = aapdhg_batch_set_tolerances(co.b, tol.data());
    if (st == AAPDHG_OK) st = aapdhg_batch_device_bytes(co.b, &co.bytes);
    if (st != AAPDHG_OK) {
        const std::string why = co.b ? aapdhg_batch_last_error(co.b) : aapdhg_batch_last_error(nullptr);
        if (co.b) aapdhg_batch_destroy(co.b);
        cudaStreamDestroy(co.stream);
        // the requests cannot be solved as given
        for (int64_t id : ids) {
            s->reqs[id].state = AAPDHG_REQ_ERROR;
            s->reqs[id].t_done = now_s(s);
        }
        if (st == AAPDHG_ERR_INVALID || st == AAPDHG_ERR_OOM) return AAPDHG_OK;
        return sfail(s, st, "cohort set-up: " + why);
    }
    const double t = now_s(s);
    for (int64_t id : ids) {
        s->reqs[id].state = AAPDHG_REQ_RUNNING;
        s->reqs[id].t_admit = t;
    }
    s->held += co.bytes;
    s->cohorts.push_back(co);
    return AAPDHG_OK;
}

// Results of a finished cohort back to its requests; its memory is freed.
aapdhg_status retire(aapdhg_server_t s, Cohort &co) {
    const int32_t k = (int32_t)co.ids.size();
    std::vector<int64_t> st6(6 * (size_t)k);
    std::vector<double> kkt(6 * (size_t)k);
    int64_t X = 0, Y = 0;
    for (int64_t id : co.ids) { X += s->reqs[id].n; Y += s->reqs[id].m; }
    std::vector<double> x(X), y(Y);
    aapdhg_status st = aapdhg_batch_get_status(co.b, st6.data());
    if (st == AAPDHG_OK) st = aapdhg_batch_get_iterate(co.b, x.data(), y.data());
    if (st == AAPDHG_OK) st = aapdhg_batch_get_kkt(co.b, kkt.data());
    const double t = now_s(s);
    int64_t xo = 0, yo = 0;
    for (int32_t i = 0; i < k; ++i) {
        Request &r = s->reqs[co.ids[i]];
        if (r.collected) {
            xo += r.n;
            yo += r.m;
            continue;
        }
        if (st == AAPDHG_OK) {
            r.x.assign(x.begin() + xo, x.begin() + xo + r.n);
            r.y.assign(y.begin() + yo, y.begin() + yo + r.m);
            for (int j = 0; j < 6; ++j) r.kkt[j] = kkt[6 * i + j];
            r.iters = st6[6 * i];
            if (st6[6 * i + 5]) r.state = AAPDHG_REQ_ERROR;
            else if (st6[6 * i + 4]) r.state = AAPDHG_REQ_CONVERGED;
            else r.state = AAPDHG_REQ_CAPPED;
        } else {
            r.state = AAPDHG_REQ_ERROR;
        }
        if (r.t_done < 0) r.t_done = t;
        xo += r.n;
        yo += r.m;
    }
    aapdhg_batch_destroy(co.b);
    cudaStreamDestroy(co.stream);
    s->held -= co.bytes;
    co.b = nullptr;
    return st == AAPDHG_OK ? AAPDHG_OK : sfail(s, st, "reading a finished cohort");
}

}  // namespace

extern "C" {

aapdhg_status aapdhg_server_create(int32_t method, int32_t m_A, int32_t max_cohorts,
                                   int32_t max_cohort_size, int64_t max_iters, int64_t mem_budget,
                                   aapdhg_server_t *out) {
    if (!out) return sfail(nullptr, AAPDHG_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (method < 0 || method > 2 || m_A < 0 || m_A > AAPDHG_MAX_MEMORY || max_cohorts < 1 ||
        max_cohort_size < 1 || max_iters < 1 || mem_budget < 0)
        return sfail(nullptr, AAPDHG_ERR_INVALID, "server parameters out of range");
    aapdhg_server_t s = new (std::nothrow) aapdhg_server_s();
    if (!s) return sfail(nullptr, AAPDHG_ERR_OOM, "host allocation");
    s->method = method;
    s->mem = m_A;
    s->max_cohorts = max_cohorts;
    s->max_cohort_size = max_cohort_size;
    s->max_iters = max_iters;
    s->budget = mem_budget;
    if (s->budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return sfail(nullptr, AAPDHG_ERR_CUDA, "cudaMemGetInfo");
        }
        s->budget = (int64_t)(0.8 * (double)fr);
    }
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return AAPDHG_OK;
}

aapdhg_status aapdhg_server_set_primal_weight(aapdhg_server_t s, int64_t period, double theta,
                                              double eps_zero, int32_t dhat_blend, double rho_min,
                                              double alpha_dec, double alpha_inc) {
    if (!s) return AAPDHG_ERR_INVALID;
    if (s->sticky) return s->sticky;
    if (period < 0 || !(theta >= 0 && theta <= 1) || !(eps_zero >= 0) || !std::isfinite(rho_min) ||
        !(alpha_dec >= 0 && alpha_dec <= 1) || !(alpha_inc >= 0 && alpha_inc <= 1)) {
        s->err = "primal weight parameters out of range";
        return AAPDHG_ERR_INVALID;                   // not sticky: the server goes on
    }
    s->pw_period = period;
    s->pw_theta = theta;
    s->pw_eps = eps_zero;
    s->pw_dhat = dhat_blend ? 1 : 0;
    s->pw_rho_min = rho_min;
    s->pw_alpha_dec = alpha_dec;
    s->pw_alpha_inc = alpha_inc;
    return AAPDHG_OK;
}

aapdhg_status aapdhg_server_submit(aapdhg_server_t s, int32_t m, int32_t n, int64_t nnz,
                                   const int64_t *row_ptr, const int32_t *col_idx, const double *val,
                                   const int8_t *row_sense, const double *q, const double *c,
                                   const double *lb, const double *ub, double tol, int64_t *id) {
    if (!s || !id) return AAPDHG_ERR_INVALID;
    if (s->sticky) return s->sticky;
    // a malformed request is refused here (not sticky: the server goes on)
    const std::string why = !(tol > 0) ? std::string("tol must be > 0")
                                       : aaph::validate_lp(m, n, nnz, row_ptr, col_idx, val,
                                                           row_sense, q, c, lb, ub);
    if (!why.empty()) {
        s->err = "request refused: " + why;
        return AAPDHG_ERR_INVALID;
    }
    Request r;
    r.m = m;
    r.n = n;
    r.rp.assign(row_ptr, row_ptr + m + 1);
    r.ci.assign(col_idx, col_idx + nnz);
    r.val.assign(val, val + nnz);
    r.sense.assign(row_sense, row_sense + m);
    r.q.assign(q, q + m);
    r.c.assign(c, c + n);
    r.lb.assign(lb, lb + n);
    r.ub.assign(ub, ub + n);
    r.tol = tol;
    r.prec = tol < s->mixed_tol_limit ? AAPDHG_FP64 : AAPDHG_MIXED;
    r.est_bytes = estimate_bytes(s, r);
    r.t_submit = now_s(s);
    *id = (int64_t)s->reqs.size();
    s->waiting[r.prec == AAPDHG_FP64 ? 1 : 0].push_back(*id);
    s->reqs.push_back(std::move(r));
    return AAPDHG_OK;
}

aapdhg_status aapdhg_server_step(aapdhg_server_t s, int32_t *running, int32_t *waiting) {
    aaph::NvtxRange range("aapdhg_server_step");
    if (!s) return AAPDHG_ERR_INVALID;
    if (s->sticky) return s->sticky;
    aapdhg_status st = AAPDHG_OK;
    // 1. one chunk on every running cohort, not waited for
    for (Cohort &co : s->cohorts) {
        const int64_t n = std::min<int64_t>(s->kkt_every, s->max_iters + 1 - co.iters);
        if (n > 0 && (st = aapdhg_batch_launch(co.b, n, 0.0, s->kkt_every)) != AAPDHG_OK)
            return sfail(s, st, std::string("launch: ") + aapdhg_batch_last_error(co.b));
        co.iters += std::max<int64_t>(n, 0);
    }
    // 2. admission while the GPU works (mixed class first, then FP64)
    for (int cls = 0; cls < 2; ++cls)
        while ((int32_t)s->cohorts.size() < s->max_cohorts && !s->waiting[cls].empty()) {
            const size_t before = s->waiting[cls].size();
            if ((st = admit(s, cls)) != AAPDHG_OK) return st;
            if (s->waiting[cls].size() == before) break;   // nothing fits now
        }
    // 3. poll; retire finished cohorts
    for (size_t i = 0; i < s->cohorts.size();) {
        Cohort &co = s->cohorts[i];
        int32_t stopped = 0;
        if (co.iters > 0) {
            if ((st = aapdhg_batch_poll(co.b, &stopped)) != AAPDHG_OK)
                return sfail(s, st, std::string("poll: ") + aapdhg_batch_last_error(co.b));
            std::vector<int64_t> st6(6 * co.ids.size());
            if ((st = aapdhg_batch_get_status(co.b, st6.data())) != AAPDHG_OK) return sfail(s, st, "status");
            const double t = now_s(s);
            for (size_t j = 0; j < co.ids.size(); ++j) {
                Request &r = s->reqs[co.ids[j]];
                if (r.collected || !(st6[6 * j + 4] || st6[6 * j + 5])) continue;
                if (r.t_done < 0) r.t_done = t;
                // the member's result now, while its cohort runs on
                r.x.resize(r.n);
                r.y.resize(r.m);
                int64_t row[6];
                if ((st = aapdhg_batch_get_member(co.b, (int32_t)j, r.x.data(), r.y.data(), r.kkt, row)) !=
                    AAPDHG_OK)
                    return sfail(s, st, std::string("member result: ") + aapdhg_batch_last_error(co.b));
                r.iters = row[0];
                r.state = row[5] ? AAPDHG_REQ_ERROR : AAPDHG_REQ_CONVERGED;
                r.collected = true;
            }
        }
        if (stopped || co.iters > s->max_iters) {
            if ((st = retire(s, co)) != AAPDHG_OK) return st;
            s->cohorts.erase(s->cohorts.begin() + (long)i);
        } else {
            ++i;
        }
    }
    if (running) *running = (int32_t)s->cohorts.size();
    if (waiting) *waiting = (int32_t)(s->waiting[0].size() + s->waiting[1].size());
    return AAPDHG_OK;
}

aapdhg_status aapdhg_server_result(aapdhg_server_t s, int64_t id, int32_t *state, double *x,
                                   double *y, double *kkt6, int64_t *iters, double *times3) {
    if (!s || id < 0 || id >= (int64_t)s->reqs.size()) return AAPDHG_ERR_INVALID;
    const Request &r = s->reqs[id];
    if (state) *state = r.state;
    if (times3) { times3[0] = r.t_submit; times3[1] = r.t_admit; times3[2] = r.t_done; }
    const bool fin = r.state == AAPDHG_REQ_CONVERGED || r.state == AAPDHG_REQ_CAPPED ||
                     (r.state == AAPDHG_REQ_ERROR && !r.x.empty());
    if (!fin) return AAPDHG_OK;
    if (x) for (int32_t j = 0; j < r.n; ++j) x[j] = r.x[j];
    if (y) for (int32_t i = 0; i < r.m; ++i) y[i] = r.y[i];
    if (kkt6) for (int j = 0; j < 6; ++j) kkt6[j] = r.kkt[j];
    if (iters) *iters = r.iters;
    return AAPDHG_OK;
}

aapdhg_status aapdhg_server_device_bytes(aapdhg_server_t s, int64_t *bytes) {
    if (!s || !bytes) return AAPDHG_ERR_INVALID;
    *bytes = s->held;
    return AAPDHG_OK;
}

const char *aapdhg_server_last_error(aapdhg_server_t s) {
    if (!s) return g_server_create_err.c_str();
    return s->err.c_str();
}

void aapdhg_server_destroy(aapdhg_server_t s) {
    if (!s) return;
    for (Cohort &co : s->cohorts) {
        if (co.b) aapdhg_batch_destroy(co.b);
        if (co.stream) cudaStreamDestroy(co.stream);
    }
    delete s;
}

}  // extern "C"
