/*
 * Plain FP64 CPU oracle of PDHG, AA-PDHG and FAA-PDHG for linear programs
 * (arXiv 2508.08062).
 *
 * TEST INFRASTRUCTURE. This file is the parity reference of the CUDA library.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load it; the product path never does, and the two share no code.
 *
 * Everything is double precision, single threaded, and written as the paper
 * states it: one loop per formula, no blocking, no fusion, no incremental
 * updates. Each function names the section, equation or algorithm it follows.
 *
 * LP form (Sec. 2.1, eq. LP-O):  min c'x  s.t.  Gx >= h,  Ax = b,  l <= x <= u.
 * K = [G; A] is passed as one CSR matrix with a per-row sense byte
 * (1 = ">=" row of G, 0 = "=" row of A), so rows of either kind may come in
 * any order; q = [h; b] likewise (eq. lambda-case).  l and u may hold -inf/+inf.
 *
 * Readings where the paper is silent or ambiguous (each also listed in the
 * design notes of the repository):
 *  R1  x^0 = P_X(0), y^0 = 0 unless a start is given (Alg. 2 only asks for a
 *      feasible start); a given start is projected onto X x Y.
 *  R2  The termination test of Alg. 2 is replaced by KKT <= tol (Remark on
 *      termination), evaluated at u^k before T(u^k) is used, every
 *      kkt_every-th loop iteration.
 *  R3  The safeguard reads ||g^k|| <= D ||g^0|| (i^k / c_div + 1)^-(1+eps);
 *      c_div = 1 is Alg. 2 exactly, c_div = 3 is the "Iter_AA / c" variant of
 *      the hyper-parameter study (real division).
 *  R4  A Cholesky failure of (dG'dG + eta I) rejects the AA step: the PDHG
 *      step is taken and counted as a fallback.
 *  R5  D-hat: the block of size n scales x and the block of size m scales y
 *      (the remark's labels "dual"/"primal" contradict the dimensions).
 *  R6  AngleFilter (Alg. 4) computes one QR before its loop; every sigma_i is
 *      read from that QR and all flagged columns are removed together.  A zero
 *      column (||f_i|| = 0) counts as sigma_i = 0.
 *  R7  LengthFilter (Alg. 5) keeps 0 columns when no k passes the test; with
 *      no kept column H^k = -beta D-hat.
 *  R8  FAA memory: adaptive mode (faa_adaptive = 1, the implemented variant of
 *      Sec. 5) replaces the memory by the filtered columns after every
 *      accepted AA step; literal mode filters a copy.
 *  R12 Preconditioning (Sec. 5.2: Ruiz scaling for 10 iterations combined with
 *      the Pock-Chambolle technique): each Ruiz pass divides every row and
 *      every column of the current scaled K by the square root of its
 *      largest |entry| (both from the same matrix; an empty row or column
 *      keeps factor 1); the Pock-Chambolle pass (alpha = 1) then divides them
 *      by the square root of their sum of |entries|.  The scaled LP is
 *      Dr K Dc, Dr q, Dc c, bounds / Dc, with x = Dc x~ and y = Dr y~.
 *  R13 Primal weight (Alg. "Primal weight update"; Remark on its form): the
 *      step sizes are tau = gamma / omega, sigma = gamma omega, so the given
 *      (tau, sigma) fix gamma = sqrt(tau sigma) and omega^0 = sqrt(sigma / tau).
 *      The update is tried when the current iterate is u^k with k > 0 and
 *      k = 0 mod U_P; Delta_x, Delta_y are the norms of the change of x and y
 *      since u^{k - U_P} (u^0 for the first), whether or not the previous try
 *      changed omega.
 *  R14 D-hat re-blend (same Remark): applied at each update that changes
 *      omega, D-hat = (1 - alpha) diag(1/omega, omega) + alpha diag(D1/omega,
 *      D2 omega) with D1, D2 the blocks of the base D-hat; r_k and r_{k-1}
 *      are the two latest residual norms ||g^{k-1}||, ||g^{k-2}||; the paper
 *      gives no threshold for a "sufficient" decrease: rho_k >= rho_min
 *      (default 0.1) selects alpha = 0.1, otherwise alpha = 0.9.  The epsilon
 *      of rho_k is epsilon_zero.
 *  R15 Memory reset: the update removes every memory column, and the pair
 *      (u^k - u^{k-1}, g^k - g^{k-1}) across it (residuals of two different
 *      operators) is not formed: that iteration takes the plain step
 *      u^{k+1} = T(u^k) with the new steps (a PDHG step, counted in j) and the
 *      memory restarts from it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t m, n;          /* rows of K (m1 + m2), columns (variables)        */
    const int64_t *rp;     /* CSR row pointers, m + 1 entries                  */
    const int32_t *ci;     /* CSR column indices                               */
    const double *v;       /* CSR values                                       */
    const int8_t *sense;   /* 1: row of G (>=), 0: row of A (=)                */
    const double *q, *c, *l, *u;
} orc_lp;

typedef struct {
    int32_t method;        /* 0 PDHG, 1 AA-PDHG (Alg. 2), 2 FAA-PDHG (Alg. 3) */
    int32_t mem;           /* m_A                                              */
    double tau, sigma;     /* step sizes of eq. pdhg                           */
    double D, eps;         /* safeguard constants                              */
    double eta;            /* Tikhonov parameter (Alg. 2 only)                 */
    double beta;           /* damping                                          */
    double c_s, kappa;     /* angle / length filter thresholds (Alg. 4, 5)     */
    double c_div;          /* safeguard divisor (R3)                           */
    int32_t dhat_mode;     /* 0: D-hat = I, 1: Remark on D-hat construction    */
    int32_t faa_adaptive;  /* R8                                               */
    /* primal weight update (Alg. "Primal weight update", Remark on its form;
     * readings R13-R15); pw_period = 0 switches it off                       */
    int32_t pw_period;     /* U_P                                              */
    double pw_theta;       /* smoothing theta                                  */
    double pw_eps_zero;    /* epsilon_zero (also the epsilon of rho_k)         */
    int32_t pw_dhat;       /* 1: re-blend D-hat at each update (Remark)        */
    double pw_rho_min;     /* "sufficient" decrease of ||g|| (R14)             */
    double pw_alpha_dec;   /* alpha when the residual decreased sufficiently   */
    double pw_alpha_inc;   /* alpha otherwise                                  */
} orc_params;

/* ------------------------------------------------------------------------ */
/* Small helpers                                                             */
/* ------------------------------------------------------------------------ */

static double dot(int64_t len, const double *a, const double *b) {
    double s = 0.0;
    for (int64_t i = 0; i < len; ++i) s += a[i] * b[i];
    return s;
}

static double clamp(double v, double lo, double hi) {
    if (v < lo) return lo;
    if (v > hi) return hi;
    return v;
}

/* (K x)_i = sum_j K_ij x_j */
static void mat_vec(const orc_lp *lp, const double *x, double *out) {
    for (int32_t i = 0; i < lp->m; ++i) {
        double s = 0.0;
        for (int64_t p = lp->rp[i]; p < lp->rp[i + 1]; ++p) s += lp->v[p] * x[lp->ci[p]];
        out[i] = s;
    }
}

/* (K' y)_j = sum_i K_ij y_i */
static void mat_t_vec(const orc_lp *lp, const double *y, double *out) {
    for (int32_t j = 0; j < lp->n; ++j) out[j] = 0.0;
    for (int32_t i = 0; i < lp->m; ++i)
        for (int64_t p = lp->rp[i]; p < lp->rp[i + 1]; ++p) out[lp->ci[p]] += lp->v[p] * y[i];
}

/* P_X and P_Y of Sec. 3: clamp x into [l, u]; y_i >= 0 on rows of G. */
static void project(const orc_lp *lp, double *x, double *y) {
    for (int32_t j = 0; j < lp->n; ++j) x[j] = clamp(x[j], lp->l[j], lp->u[j]);
    for (int32_t i = 0; i < lp->m; ++i)
        if (lp->sense[i] == 1 && y[i] < 0.0) y[i] = 0.0;
}

/* ------------------------------------------------------------------------ */
/* D-hat (Remark on the construction of D-hat), reading R5                   */
/* ------------------------------------------------------------------------ */
void orc_dhat(const orc_lp *lp, int32_t mode, double *dx, double *dy) {
    for (int32_t j = 0; j < lp->n; ++j) dx[j] = 0.0;
    for (int32_t i = 0; i < lp->m; ++i) dy[i] = 0.0;
    if (mode == 0) {
        for (int32_t j = 0; j < lp->n; ++j) dx[j] = 1.0;
        for (int32_t i = 0; i < lp->m; ++i) dy[i] = 1.0;
        return;
    }
    /* column-wise and row-wise max |K_ij| */
    for (int32_t i = 0; i < lp->m; ++i)
        for (int64_t p = lp->rp[i]; p < lp->rp[i + 1]; ++p) {
            double a = fabs(lp->v[p]);
            if (a > dx[lp->ci[p]]) dx[lp->ci[p]] = a;
            if (a > dy[i]) dy[i] = a;
        }
    for (int32_t j = 0; j < lp->n; ++j) dx[j] = sqrt(fmax(dx[j], 1e-10));
    for (int32_t i = 0; i < lp->m; ++i) dy[i] = sqrt(fmax(dy[i], 1e-10));
}

/* ------------------------------------------------------------------------ */
/* Diagonal preconditioning factors (reading R12): dr (m), dc (n).           */
/* ------------------------------------------------------------------------ */
static void scaled_row_col(const orc_lp *lp, const double *dr, const double *dc, int sum,
                           double *rn, double *cn) {
    for (int32_t i = 0; i < lp->m; ++i) rn[i] = 0.0;
    for (int32_t j = 0; j < lp->n; ++j) cn[j] = 0.0;
    for (int32_t i = 0; i < lp->m; ++i)
        for (int64_t p = lp->rp[i]; p < lp->rp[i + 1]; ++p) {
            const int32_t j = lp->ci[p];
            const double a = fabs(dr[i] * lp->v[p] * dc[j]);
            if (sum) { rn[i] += a; cn[j] += a; }
            else { if (a > rn[i]) rn[i] = a; if (a > cn[j]) cn[j] = a; }
        }
}

void orc_scaling(const orc_lp *lp, int32_t ruiz_iters, int32_t pock_chambolle, double *dr,
                 double *dc) {
    double *rn = calloc(lp->m > 0 ? lp->m : 1, sizeof(double));
    double *cn = calloc(lp->n > 0 ? lp->n : 1, sizeof(double));
    for (int32_t i = 0; i < lp->m; ++i) dr[i] = 1.0;
    for (int32_t j = 0; j < lp->n; ++j) dc[j] = 1.0;
    for (int32_t pass = 0; pass < ruiz_iters + (pock_chambolle ? 1 : 0); ++pass) {
        const int sum = pass >= ruiz_iters;      /* the last pass is Pock-Chambolle */
        scaled_row_col(lp, dr, dc, sum, rn, cn);
        for (int32_t i = 0; i < lp->m; ++i) if (rn[i] > 0.0) dr[i] /= sqrt(rn[i]);
        for (int32_t j = 0; j < lp->n; ++j) if (cn[j] > 0.0) dc[j] /= sqrt(cn[j]);
    }
    free(rn); free(cn);
}

/* ------------------------------------------------------------------------ */
/* The PDHG map T (Sec. 3, eq. pdhg; fixed-point form eq. new-fixed-point)   */
/*   xh = P_X(x - tau (c - K'y))                                            */
/*   yh = P_Y(y + sigma (q - K(2 xh - x)))                                  */
/* ------------------------------------------------------------------------ */
void orc_T(const orc_lp *lp, double tau, double sigma, const double *x, const double *y,
           double *xh, double *yh) {
    int32_t m = lp->m, n = lp->n;
    double *kty = calloc(n > 0 ? n : 1, sizeof(double));
    double *z = calloc(n > 0 ? n : 1, sizeof(double));
    double *kz = calloc(m > 0 ? m : 1, sizeof(double));
    mat_t_vec(lp, y, kty);
    for (int32_t j = 0; j < n; ++j) xh[j] = clamp(x[j] - tau * (lp->c[j] - kty[j]), lp->l[j], lp->u[j]);
    for (int32_t j = 0; j < n; ++j) z[j] = 2.0 * xh[j] - x[j];
    mat_vec(lp, z, kz);
    for (int32_t i = 0; i < m; ++i) {
        double v = y[i] + sigma * (lp->q[i] - kz[i]);
        if (lp->sense[i] == 1 && v < 0.0) v = 0.0;
        yh[i] = v;
    }
    free(kty); free(z); free(kz);
}

/* ------------------------------------------------------------------------ */
/* KKT residuals (Remark on termination conditions; Lambda from eq.          */
/* lambda-case).  out = {r_p, r_d, r_g, KKT, pobj, dobj}                      */
/* ------------------------------------------------------------------------ */
void orc_kkt(const orc_lp *lp, const double *x, const double *y, double *out) {
    int32_t m = lp->m, n = lp->n;
    double *kx = malloc(sizeof(double) * (m > 0 ? m : 1));
    double *kty = malloc(sizeof(double) * (n > 0 ? n : 1));
    mat_vec(lp, x, kx);
    mat_t_vec(lp, y, kty);

    /* primal infeasibility: (b - Ax) on "=" rows, (h - Gx)_+ on ">=" rows */
    double pres2 = 0.0, qn2 = 0.0, qty = 0.0;
    for (int32_t i = 0; i < m; ++i) {
        double r = lp->q[i] - kx[i];
        if (lp->sense[i] == 1) r = r > 0.0 ? r : 0.0;
        pres2 += r * r;
        qn2 += lp->q[i] * lp->q[i];
        qty += lp->q[i] * y[i];
    }

    /* lambda = P_Lambda(c - K'y); Lambda_j by finiteness of l_j, u_j */
    double dres2 = 0.0, cn2 = 0.0, ctx = 0.0, lam_terms = 0.0;
    for (int32_t j = 0; j < n; ++j) {
        double r = lp->c[j] - kty[j];
        int lo_fin = isfinite(lp->l[j]), up_fin = isfinite(lp->u[j]);
        double lam;
        if (!lo_fin && !up_fin) lam = 0.0;                 /* {0}  */
        else if (!lo_fin && up_fin) lam = r < 0.0 ? r : 0.0; /* R_-  */
        else if (lo_fin && !up_fin) lam = r > 0.0 ? r : 0.0; /* R_+  */
        else lam = r;                                       /* R    */
        double d = r - lam;
        dres2 += d * d;
        cn2 += lp->c[j] * lp->c[j];
        ctx += lp->c[j] * x[j];
        /* l' lambda+ - u' lambda-, lambda+ = max(lambda, 0), lambda- = max(-lambda, 0) */
        if (lam > 0.0) lam_terms += lp->l[j] * lam;
        if (lam < 0.0) lam_terms -= lp->u[j] * (-lam);
    }
    double dobj = qty + lam_terms;
    double pobj = ctx;
    double r_p = sqrt(pres2) / (1.0 + sqrt(qn2));
    double r_d = sqrt(dres2) / (1.0 + sqrt(cn2));
    double r_g = fabs(dobj - pobj) / (1.0 + fabs(dobj) + fabs(pobj));
    double kkt = r_p;
    if (r_d > kkt) kkt = r_d;
    if (r_g > kkt) kkt = r_g;
    out[0] = r_p; out[1] = r_d; out[2] = r_g; out[3] = kkt; out[4] = pobj; out[5] = dobj;
    free(kx); free(kty);
}

/* ------------------------------------------------------------------------ */
/* Dense helpers for the Anderson subproblems.  Matrices are column-major,  */
/* column j of an N x k matrix A starting at A + j*N.                        */
/* ------------------------------------------------------------------------ */

/* Cholesky S = L L' of a k x k symmetric matrix (row-major).  Returns 0 on
 * success, -1 when a pivot is not positive.                                  */
static int cholesky(int k, const double *S, double *L) {
    memset(L, 0, sizeof(double) * k * k);
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = S[i * k + j];
            for (int p = 0; p < j; ++p) s -= L[i * k + p] * L[j * k + p];
            if (i == j) {
                if (!(s > 0.0)) return -1;
                L[i * k + i] = sqrt(s);
            } else {
                L[i * k + j] = s / L[j * k + j];
            }
        }
    }
    return 0;
}

/* gamma = (dG' dG + eta I)^-1 dG' g  (the Tikhonov-regularised least-squares
 * factor of H^k in Alg. 2).  dG is N x k column-major.  Returns 0, or -1 when
 * the Cholesky factorisation fails (reading R4).                              */
int orc_aa_coeffs(int64_t N, int32_t k, const double *dG, const double *g, double eta,
                  double *gamma) {
    if (k <= 0) return 0;
    double *S = malloc(sizeof(double) * k * k);
    double *L = malloc(sizeof(double) * k * k);
    double *rhs = malloc(sizeof(double) * k);
    for (int a = 0; a < k; ++a) {
        for (int b = 0; b < k; ++b) S[a * k + b] = dot(N, dG + (int64_t)a * N, dG + (int64_t)b * N);
        S[a * k + a] += eta;
        rhs[a] = dot(N, dG + (int64_t)a * N, g);
    }
    int rc = cholesky(k, S, L);
    if (rc == 0) {
        /* forward solve L w = rhs, back solve L' gamma = w */
        for (int i = 0; i < k; ++i) {
            double s = rhs[i];
            for (int p = 0; p < i; ++p) s -= L[i * k + p] * gamma[p];
            gamma[i] = s / L[i * k + i];
        }
        for (int i = k - 1; i >= 0; --i) {
            double s = gamma[i];
            for (int p = i + 1; p < k; ++p) s -= L[p * k + i] * gamma[p];
            gamma[i] = s / L[i * k + i];
        }
    }
    free(S); free(L); free(rhs);
    return rc;
}

/* The Anderson step before the projection (Alg. 2, AA branch):
 *     u_AA = u^k - H^k g^k,   H^k = -beta D-hat + (dU + beta D-hat dG) (dG'dG + eta I)^-1 dG',
 * so with gamma = (dG'dG + eta I)^-1 dG'g^k (orc_aa_coeffs, or the FAA solve)
 *     u_AA = u^k + beta D-hat g^k - (dU + beta D-hat dG) gamma.
 * E = dU and F = dG are N x k column-major; dh is the diagonal of D-hat.
 * The projection P onto X x Y is applied by the caller.                      */
void orc_aa_mix(int64_t N, int32_t k, const double *u, const double *g, const double *E,
                const double *F, const double *dh, double beta, const double *gamma,
                double *out) {
    for (int64_t e = 0; e < N; ++e) {
        double s = 0.0;
        for (int j = 0; j < k; ++j)
            s += (E[(int64_t)j * N + e] + beta * dh[e] * F[(int64_t)j * N + e]) * gamma[j];
        out[e] = u[e] + beta * dh[e] * g[e] - s;
    }
}

/* Economy QR by Householder reflections of an N x k column-major matrix F.
 * On return R (k x k, row-major, upper triangular) holds the R factor and, if
 * qtb is given, qtb = Q' b for the vector b.  Signs of R's rows follow the
 * reflections; only |r_ii| and R^-1 Q' b are used, both sign-independent.    */
static void householder_qr(int64_t N, int k, const double *F, double *R, const double *b,
                           double *qtb) {
    double *A = malloc(sizeof(double) * (N * k > 0 ? N * k : 1));
    double *w = malloc(sizeof(double) * (N > 0 ? N : 1));
    double *bb = NULL;
    memcpy(A, F, sizeof(double) * N * k);
    if (b) { bb = malloc(sizeof(double) * (N > 0 ? N : 1)); memcpy(bb, b, sizeof(double) * N); }
    memset(R, 0, sizeof(double) * k * k);
    for (int j = 0; j < k && j < N; ++j) {
        double *a = A + (int64_t)j * N;
        double norm = 0.0;
        for (int64_t i = j; i < N; ++i) norm += a[i] * a[i];
        norm = sqrt(norm);
        if (norm > 0.0) {
            double alpha = a[j] > 0.0 ? -norm : norm;   /* reflect a[j:] onto alpha e_j */
            for (int64_t i = 0; i < N; ++i) w[i] = (i < j) ? 0.0 : a[i];
            w[j] -= alpha;
            double wn2 = 0.0;
            for (int64_t i = j; i < N; ++i) wn2 += w[i] * w[i];
            if (wn2 > 0.0) {
                for (int c = j; c < k; ++c) {
                    double *col = A + (int64_t)c * N;
                    double s = 0.0;
                    for (int64_t i = j; i < N; ++i) s += w[i] * col[i];
                    s = 2.0 * s / wn2;
                    for (int64_t i = j; i < N; ++i) col[i] -= s * w[i];
                }
                if (bb) {
                    double s = 0.0;
                    for (int64_t i = j; i < N; ++i) s += w[i] * bb[i];
                    s = 2.0 * s / wn2;
                    for (int64_t i = j; i < N; ++i) bb[i] -= s * w[i];
                }
            }
        }
        for (int c = j; c < k; ++c) R[j * k + c] = A[(int64_t)c * N + j];
    }
    if (qtb) for (int j = 0; j < k; ++j) qtb[j] = (j < N) ? bb[j] : 0.0;
    free(A); free(w); free(bb);
}

/* gamma = R^-1 Q' g with dG = QR (Alg. 3, eq. AA-update_filter1).  Returns 0,
 * or -1 when R has a zero diagonal entry.                                    */
int orc_qr_coeffs(int64_t N, int32_t k, const double *dG, const double *g, double *gamma) {
    if (k <= 0) return 0;
    double *R = malloc(sizeof(double) * k * k);
    double *qtg = malloc(sizeof(double) * k);
    householder_qr(N, k, dG, R, g, qtg);
    int rc = 0;
    for (int i = k - 1; i >= 0; --i) {
        double s = qtg[i];
        for (int p = i + 1; p < k; ++p) s -= R[i * k + p] * gamma[p];
        if (R[i * k + i] == 0.0) { rc = -1; break; }
        gamma[i] = s / R[i * k + i];
    }
    free(R); free(qtg);
    return rc;
}

/* Upper bounds b_j on ||column j of R^-1||^2 (Lemma "Proposition 1.2" of
 * Sec. 4), j = 1..k, from the column norms fn[] of F and c_s.                */
void orc_length_bounds(int32_t k, const double *fn, double c_s, double *b) {
    double c_t = sqrt(1.0 - c_s * c_s);
    for (int j = 1; j <= k; ++j) {
        double fj2 = fn[j - 1] * fn[j - 1];
        if (j == 1) { b[0] = 1.0 / fj2; continue; }
        double f12 = fn[0] * fn[0];
        double s = c_t * c_t * pow(c_t + c_s, 2.0 * (j - 2)) / (f12 * pow(c_s, 2.0 * (j - 2)));
        for (int i = 2; i <= j - 1; ++i) {
            double fi2 = fn[i - 1] * fn[i - 1];
            s += c_t * c_t * pow(c_t + c_s, 2.0 * (j - i - 1)) / (fi2 * pow(c_s, 2.0 * (j - i)));
        }
        s += 1.0 / fj2;
        b[j - 1] = s / (c_s * c_s);
    }
}

/* Reverse (Alg. 6), AngleFilter (Alg. 4), LengthFilter (Alg. 5), Reverse.
 * Input: E = dU and F = dG, N x k column-major, oldest column first.
 * Output: keep[j] = 1 for the columns (oldest-first indexing) that survive.
 * Returns the number of kept columns.                                        */
int32_t orc_faa_filter(int64_t N, int32_t k, const double *E, const double *F, double c_s,
                       double kappa, int32_t *keep) {
    if (k <= 0) return 0;
    for (int j = 0; j < k; ++j) keep[j] = 0;
    /* Reverse: newest column first */
    double *Fr = malloc(sizeof(double) * N * k);
    int *orig = malloc(sizeof(int) * k);      /* reversed position -> oldest-first index */
    for (int j = 0; j < k; ++j) {
        orig[j] = k - 1 - j;
        memcpy(Fr + (int64_t)j * N, F + (int64_t)orig[j] * N, sizeof(double) * N);
    }
    /* AngleFilter: one economy QR, sigma_i = |r_ii| / ||f_i||, i = 2..k (R6) */
    double *R = malloc(sizeof(double) * k * k);
    householder_qr(N, k, Fr, R, NULL, NULL);
    int *alive = malloc(sizeof(int) * k);
    alive[0] = 1;
    for (int i = 1; i < k; ++i) {
        double fn = sqrt(dot(N, Fr + (int64_t)i * N, Fr + (int64_t)i * N));
        double sig = fn > 0.0 ? fabs(R[i * k + i]) / fn : 0.0;
        alive[i] = !(sig < c_s);
    }
    /* LengthFilter over the surviving columns, still newest first */
    int kk = 0;
    int *pos = malloc(sizeof(int) * k);       /* filtered position -> reversed position */
    for (int i = 0; i < k; ++i) if (alive[i]) pos[kk++] = i;
    double *en = malloc(sizeof(double) * kk), *fn = malloc(sizeof(double) * kk);
    double *b = malloc(sizeof(double) * (kk > 0 ? kk : 1));
    for (int t = 0; t < kk; ++t) {
        const double *e = E + (int64_t)orig[pos[t]] * N;
        const double *f = Fr + (int64_t)pos[t] * N;
        en[t] = sqrt(dot(N, e, e));
        fn[t] = sqrt(dot(N, f, f));
    }
    orc_length_bounds(kk, fn, c_s, b);
    int mbar = 0;                              /* R7: 0 when no prefix passes */
    for (int t = kk; t >= 1; --t) {
        double se = 0.0, sb = 0.0;
        for (int j = 0; j < t; ++j) { se += en[j] * en[j]; sb += b[j]; }
        double C = se * sb;
        if (C <= kappa * kappa) { mbar = t; break; }
    }
    /* first mbar filtered columns survive; Reverse maps them back */
    for (int t = 0; t < mbar; ++t) keep[orig[pos[t]]] = 1;
    free(Fr); free(orig); free(R); free(alive); free(pos); free(en); free(fn); free(b);
    return mbar;
}

/* ------------------------------------------------------------------------ */
/* The solver loop: PDHG, AA-PDHG (Alg. 2) and FAA-PDHG (Alg. 3).            */
/* ------------------------------------------------------------------------ */

/* trace: per loop iteration t (k = t + 1), if the arrays are given:
 *   branch[t] = 0 PDHG step (safeguard failed or method 0), 1 AA step,
 *               2 AA rejected because the LS factorisation failed (R4)
 *   gnorm[t]  = ||g^k||,   kkt[t] = KKT(u^k) or NaN when not evaluated,
 *   mk[t]     = columns used by the accepted AA step, -1 otherwise.
 * rec_u: u^1 .. u^rec_len, each (x; y), n + m doubles.
 * counters = {AA steps i, PDHG steps j, loop iterations}.
 * Returns 0 when KKT <= tol was reached, 1 when max_iters ran out.           */
int orc_solve(const orc_lp *lp, const orc_params *p, const double *x0, const double *y0,
              int64_t max_iters, double tol, int32_t kkt_every, double *x_out, double *y_out,
              int64_t *counters, int64_t trace_len, int8_t *tr_branch, double *tr_gnorm,
              double *tr_kkt, int32_t *tr_mk, int64_t rec_len, double *rec_u, double *dh_out) {
    const int32_t m = lp->m, n = lp->n;
    const int64_t N = (int64_t)n + m;
    const int M = p->method == 0 ? 0 : p->mem;
    double *u = calloc(N + 1, sizeof(double));       /* u^k = (x; y)            */
    double *u_prev = calloc(N + 1, sizeof(double));  /* u^{k-1}                 */
    double *uh = calloc(N + 1, sizeof(double));      /* T(u^k)                  */
    double *g = calloc(N + 1, sizeof(double));       /* g^k                     */
    double *g_prev = calloc(N + 1, sizeof(double));  /* g^{k-1}                 */
    double *dh = calloc(N + 1, sizeof(double));      /* D-hat                   */
    double *dU = calloc(N * (M > 0 ? M : 1) + 1, sizeof(double)); /* oldest first */
    double *dG = calloc(N * (M > 0 ? M : 1) + 1, sizeof(double));
    double *gam = calloc(M + 1, sizeof(double));
    int32_t *keep = calloc(M + 1, sizeof(int32_t));
    double *E2 = calloc(N * (M > 0 ? M : 1) + 1, sizeof(double));
    double *F2 = calloc(N * (M > 0 ? M : 1) + 1, sizeof(double));
    int cols = 0;

    orc_dhat(lp, p->dhat_mode, dh, dh + n);
    /* primal weight state (R13): gamma, omega, current steps, base D-hat,
     * the iterate at the last update point, the two latest residual norms */
    const double pw_gamma = sqrt(p->tau * p->sigma);
    double omega = sqrt(p->sigma / p->tau), tau_c = p->tau, sigma_c = p->sigma;
    double *dh_base = calloc(N + 1, sizeof(double));
    double *snap = calloc(N + 1, sizeof(double));
    memcpy(dh_base, dh, sizeof(double) * N);
    double gn_last = NAN, gn_last2 = NAN;

    /* u^0 (R1) and u^1 = T u^0, g^0 = u^1 - u^0 */
    for (int32_t j = 0; j < n; ++j) u_prev[j] = x0 ? x0[j] : 0.0;
    for (int32_t i = 0; i < m; ++i) u_prev[n + i] = y0 ? y0[i] : 0.0;
    project(lp, u_prev, u_prev + n);
    memcpy(snap, u_prev, sizeof(double) * N);
    orc_T(lp, tau_c, sigma_c, u_prev, u_prev + n, u, u + n);
    for (int64_t e = 0; e < N; ++e) g_prev[e] = u[e] - u_prev[e];
    const double g0 = sqrt(dot(N, g_prev, g_prev));
    gn_last = g0;

    int64_t i_aa = 0, j_pd = 0, it = 0;
    int status = 1;
    if (rec_len > 0) memcpy(rec_u, u, sizeof(double) * N);

    for (int64_t k = 1; it < max_iters; ++k) {
        double kk[6];
        int have_kkt = 0;
        if (kkt_every > 0 && (k - 1) % kkt_every == 0) {
            orc_kkt(lp, u, u + n, kk);
            have_kkt = 1;
            if (kk[3] <= tol) { status = 0; }
        }
        if (it < trace_len && tr_kkt) tr_kkt[it] = have_kkt ? kk[3] : NAN;
        if (status == 0) break;

        /* primal weight update (Alg. "Primal weight update"; R13-R15) */
        int restart = 0;
        if (p->pw_period > 0 && k % p->pw_period == 0) {
            double dx = 0.0, dy = 0.0;
            for (int32_t j = 0; j < n; ++j) dx += (u[j] - snap[j]) * (u[j] - snap[j]);
            for (int32_t i = 0; i < m; ++i) dy += (u[n + i] - snap[n + i]) * (u[n + i] - snap[n + i]);
            dx = sqrt(dx);
            dy = sqrt(dy);
            memcpy(snap, u, sizeof(double) * N);
            if (dx > p->pw_eps_zero && dy > p->pw_eps_zero) {
                omega = exp(p->pw_theta * log(dy / dx) + (1.0 - p->pw_theta) * log(omega));
                tau_c = pw_gamma / omega;
                sigma_c = pw_gamma * omega;
                cols = 0;                                   /* reset the memory (R15) */
                restart = 1;
                if (p->pw_dhat) {                           /* D-hat re-blend (R14) */
                    const double r1 = gn_last, r2 = gn_last2;
                    const double rho = isnan(r2) ? 0.0 : (r2 - r1) / fmax(r2, p->pw_eps_zero);
                    const double a = rho >= p->pw_rho_min ? p->pw_alpha_dec : p->pw_alpha_inc;
                    for (int32_t j = 0; j < n; ++j) dh[j] = ((1.0 - a) + a * dh_base[j]) / omega;
                    for (int32_t i = 0; i < m; ++i) dh[n + i] = ((1.0 - a) + a * dh_base[n + i]) * omega;
                }
            }
        }

        /* u-hat^{k+1} = T u^k, g^k = u-hat^{k+1} - u^k */
        orc_T(lp, tau_c, sigma_c, u, u + n, uh, uh + n);
        for (int64_t e = 0; e < N; ++e) g[e] = uh[e] - u[e];
        const double gn = sqrt(dot(N, g, g));
        gn_last2 = gn_last;
        gn_last = gn;

        /* memory update: append (u^k - u^{k-1}, g^k - g^{k-1}); keep at most m_A */
        if (M > 0 && !restart) {
            if (cols == M) {
                memmove(dU, dU + N, sizeof(double) * N * (M - 1));
                memmove(dG, dG + N, sizeof(double) * N * (M - 1));
                cols = M - 1;
            }
            for (int64_t e = 0; e < N; ++e) {
                dU[(int64_t)cols * N + e] = u[e] - u_prev[e];
                dG[(int64_t)cols * N + e] = g[e] - g_prev[e];
            }
            cols += 1;
        }

        int branch = 0, used = -1;
        double thresh = p->D * g0 * pow(i_aa / p->c_div + 1.0, -(1.0 + p->eps));
        if (p->method != 0 && M > 0 && !restart && gn <= thresh) {
            const double *Eu = dU, *Fg = dG;
            int kc = cols, rc;
            if (p->method == 1) {
                rc = orc_aa_coeffs(N, kc, Fg, g, p->eta, gam);
            } else {
                orc_faa_filter(N, kc, dU, dG, p->c_s, p->kappa, keep);
                int t = 0;
                for (int j = 0; j < kc; ++j)
                    if (keep[j]) {
                        memcpy(E2 + (int64_t)t * N, dU + (int64_t)j * N, sizeof(double) * N);
                        memcpy(F2 + (int64_t)t * N, dG + (int64_t)j * N, sizeof(double) * N);
                        ++t;
                    }
                kc = t; Eu = E2; Fg = F2;
                rc = orc_qr_coeffs(N, kc, Fg, g, gam);
                if (rc == 0 && p->faa_adaptive) {
                    memcpy(dU, E2, sizeof(double) * N * kc);
                    memcpy(dG, F2, sizeof(double) * N * kc);
                    cols = kc;
                }
            }
            if (rc == 0) {
                /* u^{k+1} = P(u^k - H^k g^k); uh is reused for u_AA */
                orc_aa_mix(N, kc, u, g, Eu, Fg, dh, p->beta, gam, uh);
                project(lp, uh, uh + n);
                branch = 1; used = kc;
            } else {
                branch = 2;
            }
        }
        if (branch == 1) i_aa += 1; else j_pd += 1;

        if (it < trace_len) {
            if (tr_branch) tr_branch[it] = (int8_t)branch;
            if (tr_gnorm) tr_gnorm[it] = gn;
            if (tr_mk) tr_mk[it] = used;
        }
        /* advance: u^{k-1} <- u^k, u^k <- u^{k+1}, g^{k-1} <- g^k */
        double *tmp = u_prev; u_prev = u; u = uh; uh = tmp;
        memcpy(g_prev, g, sizeof(double) * N);
        it += 1;
        if (it < rec_len) memcpy(rec_u + it * N, u, sizeof(double) * N);
    }

    memcpy(x_out, u, sizeof(double) * n);
    memcpy(y_out, u + n, sizeof(double) * m);
    counters[0] = i_aa; counters[1] = j_pd; counters[2] = it;
    if (dh_out) memcpy(dh_out, dh, sizeof(double) * N);   /* D-hat in use at the end */
    free(u); free(u_prev); free(uh); free(g); free(g_prev); free(dh); free(dU); free(dG);
    free(gam); free(keep); free(E2); free(F2); free(dh_base); free(snap);
    return status;
}
