/*
 * fr_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see fr_oracle.h).
 *
 * Source: Uehara et al., arXiv 2406.10262. Each function cites the passage it restates.
 * Equation numbers follow the paper's LaTeX: Eqs. (1)-(3) the doubly-stochastic constraints,
 * Eq. (4) item impact, Eq. (5) the NSW objective F, Problem (6) the fair ranking problem,
 * Problem (7) the entropic optimal-transport problem, Problem (8) the unconstrained
 * reformulation over costs C, Theorem 1, Algorithm 1, Sec. 4.1 the evaluation metrics.
 *
 * Pins (each checked by a `-m "not gpu"` test against something other than this file):
 *   orc_marginals       dummy-column mass and padded exposure: closed form (Sec. 2)
 *   orc_sinkhorn        uniform policy from C = 0 (closed form); Theorem 1 round trip; gauge
 *                       invariance; geometric convergence of the column residual; agreement with
 *                       a primal-dual gap of Problem (7) at convergence
 *   impacts / F         uniform-policy closed form; brute force over permutation mixtures
 *   orc_implicit_grad   central finite differences of F(X*(C)) at convergence; zero row and
 *                       column sums (gauge invariance of Problem (7))
 *   orc_unrolled_grad   torch.autograd in float64 through an independent restatement; finite
 *                       differences of the exact L-step map
 *   orc_adam / orc_sgd  torch.optim.Adam(maximize=True) / torch.optim.SGD in float64
 *   orc_step/orc_solve  monotone ascent under small-step SGD; F -> F* of brute force on tiny
 *                       instances; certificate >= F* - F; the stop rule of Algorithm 1: one step
 *                       when the uniform policy is optimal (|U| = 1, separable r), every step at
 *                       t = 0, and exactly j steps for a threshold between the j-th gradient norm
 *                       and the smaller earlier ones (brute-force instances); the traced norm is
 *                       that of orc_grad before the step
 *   orc_grad (omega)    central differences of sum_i omega_i Imp_i for a random omega, both
 *                       gradient modes, free costs and per-item variables, and in r
 *   orc_metrics         utility identity; envy and better/worse-off against brute force at the
 *                       optimum (envy-freeness, dominance over uniform) on small cases
 *   orc_certificate     bound checked against brute-force F*
 */
#include "fr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX3(u, i, k, I, m) (((int64_t)(u) * (I) + (i)) * (m) + (k))

static double* dalloc(int64_t n) {
    double* p = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    return p;
}

/* log(sum_j exp(v_j)) with the exact max shift. */
static double lse(const double* v, int32_t n) {
    double mx = -INFINITY;
    for (int32_t j = 0; j < n; ++j)
        if (v[j] > mx) mx = v[j];
    if (mx == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (int32_t j = 0; j < n; ++j) s += exp(v[j] - mx);
    return mx + log(s);
}

/* ---- Sec. 2: columns and marginals ----------------------------------------------------------
 * Eq. (1): every item's row sums to 1. Eq. (2): each real slot k < K receives mass 1. The last
 * (dummy) position receives I - K so that the I rows can be placed; when I == K that mass is
 * zero and the column is dropped, leaving a square doubly-stochastic matrix. */
int32_t orc_num_cols(int32_t I, int32_t K) { return I > K ? K + 1 : K; }

void orc_marginals(int32_t I, int32_t K, const double* e_in, double* b, double* e) {
    int32_t m = orc_num_cols(I, K);
    for (int32_t k = 0; k < K; ++k) {
        b[k] = 1.0;
        e[k] = e_in[k];
    }
    if (m > K) {
        b[K] = (double)(I - K);
        e[K] = 0.0; /* Eq. (4) sums over k in [m-1] only */
    }
}

/* ---- Sec. 3, Problem (7): Sinkhorn in the log domain (Cuturi 2013) ---------------------------
 * Dual potentials f (rows) and g (columns); the solution has x_ik = exp((f_i + g_k - c_ik)/eps).
 * Iteration l: row update   f_i = eps log a_i - eps LSE_k((g_k - c_ik)/eps),  a_i = 1 (Eq. 1)
 *              column update g_k = eps log b_k - eps LSE_i((f_i - c_ik)/eps)  (Eq. 2 + dummy)
 * The emitted policy is the one right after the last row update, so Eq. (1) holds exactly and
 * the column residual measures the remaining error; g^(L) is returned for warm starts. */
void orc_sinkhorn(int32_t I, int32_t m, const double* c, const double* b, double eps, int32_t L,
                  double* g, double* x, double* gprev) {
    double* f = dalloc(I);
    double* gl = dalloc(m);
    double* buf = dalloc(I > m ? I : m);
    for (int32_t l = 1; l <= L; ++l) {
        memcpy(gl, g, sizeof(double) * (size_t)m); /* g^(l-1) */
        for (int32_t i = 0; i < I; ++i) {
            for (int32_t k = 0; k < m; ++k) buf[k] = (g[k] - c[(int64_t)i * m + k]) / eps;
            f[i] = -eps * lse(buf, m);
        }
        for (int32_t k = 0; k < m; ++k) {
            for (int32_t i = 0; i < I; ++i) buf[i] = (f[i] - c[(int64_t)i * m + k]) / eps;
            g[k] = eps * log(b[k]) - eps * lse(buf, I);
        }
    }
    for (int32_t i = 0; i < I; ++i)
        for (int32_t k = 0; k < m; ++k)
            x[(int64_t)i * m + k] = exp((f[i] + gl[k] - c[(int64_t)i * m + k]) / eps);
    if (gprev) memcpy(gprev, gl, sizeof(double) * (size_t)m);
    free(f);
    free(gl);
    free(buf);
}

/* Per-item parametrisation of the cost (a structured instance of Problem (8)'s C):
 * c_ik = -r_ui e_k w_i with w_i = exp(theta_i); the dummy column (e = 0) costs 0. */
void orc_cost_item(int32_t I, int32_t m, const double* r_u, const double* e, const double* theta,
                   double* c) {
    for (int32_t i = 0; i < I; ++i) {
        double w = exp(theta[i]);
        for (int32_t k = 0; k < m; ++k) c[(int64_t)i * m + k] = -r_u[i] * e[k] * w;
    }
}

/* Solve A y = rhs (n x n, row-major, A overwritten) by Cholesky; falls back to LU with partial
 * pivoting when a pivot is not positive. Returns 0 on success. */
static int solve_spd(int32_t n, double* A, double* rhs) {
    if (n == 0) return 0;
    double* Lm = dalloc((int64_t)n * n);
    int ok = 1;
    for (int32_t j = 0; j < n && ok; ++j) {
        double d = A[(int64_t)j * n + j];
        for (int32_t p = 0; p < j; ++p) d -= Lm[(int64_t)j * n + p] * Lm[(int64_t)j * n + p];
        if (!(d > 0.0)) {
            ok = 0;
            break;
        }
        double ljj = sqrt(d);
        Lm[(int64_t)j * n + j] = ljj;
        for (int32_t i = j + 1; i < n; ++i) {
            double s = A[(int64_t)i * n + j];
            for (int32_t p = 0; p < j; ++p) s -= Lm[(int64_t)i * n + p] * Lm[(int64_t)j * n + p];
            Lm[(int64_t)i * n + j] = s / ljj;
        }
    }
    if (ok) {
        for (int32_t i = 0; i < n; ++i) { /* forward: L y = rhs */
            double s = rhs[i];
            for (int32_t p = 0; p < i; ++p) s -= Lm[(int64_t)i * n + p] * rhs[p];
            rhs[i] = s / Lm[(int64_t)i * n + i];
        }
        for (int32_t i = n - 1; i >= 0; --i) { /* backward: L^T z = y */
            double s = rhs[i];
            for (int32_t p = i + 1; p < n; ++p) s -= Lm[(int64_t)p * n + i] * rhs[p];
            rhs[i] = s / Lm[(int64_t)i * n + i];
        }
        free(Lm);
        return 0;
    }
    free(Lm);
    /* LU with partial pivoting */
    for (int32_t j = 0; j < n; ++j) {
        int32_t piv = j;
        for (int32_t i = j + 1; i < n; ++i)
            if (fabs(A[(int64_t)i * n + j]) > fabs(A[(int64_t)piv * n + j])) piv = i;
        if (A[(int64_t)piv * n + j] == 0.0) return 1;
        if (piv != j) {
            for (int32_t p = 0; p < n; ++p) {
                double tmp = A[(int64_t)j * n + p];
                A[(int64_t)j * n + p] = A[(int64_t)piv * n + p];
                A[(int64_t)piv * n + p] = tmp;
            }
            double tmp = rhs[j];
            rhs[j] = rhs[piv];
            rhs[piv] = tmp;
        }
        for (int32_t i = j + 1; i < n; ++i) {
            double f = A[(int64_t)i * n + j] / A[(int64_t)j * n + j];
            for (int32_t p = j; p < n; ++p) A[(int64_t)i * n + p] -= f * A[(int64_t)j * n + p];
            rhs[i] -= f * rhs[j];
        }
    }
    for (int32_t i = n - 1; i >= 0; --i) {
        double s = rhs[i];
        for (int32_t p = i + 1; p < n; ++p) s -= A[(int64_t)i * n + p] * rhs[p];
        rhs[i] = s / A[(int64_t)i * n + i];
    }
    return 0;
}

/* Sec. 3 (after Theorem 1): gradient of F(X*(C)) with respect to C through the chain rule, where
 * the derivative of X*(C) comes from the optimality conditions of Problem (7). At the solution x_ik = exp((f_i + g_k - c_ik)/eps), so a
 * cost perturbation moves x by x_ik (df_i + dg_k - dc_ik)/eps while the marginals stay fixed.
 * Eliminating df, dg with multipliers alpha (rows) and beta (columns):
 *     h_i = sum_k x_ik gx_ik,  q_k = sum_i x_ik gx_ik,  cs_k = sum_i x_ik,
 *     (diag(cs) - X^T X) beta = q - X^T h   (singular along 1: beta_{m-1} := 0),
 *     alpha_i = h_i - sum_k x_ik beta_k,
 *     dF/dc_ik = -(1/eps) x_ik (gx_ik - alpha_i - beta_k).
 * Rows of x sum to 1 (the emitted policy), which the elimination uses. */
void orc_implicit_grad(int32_t I, int32_t m, const double* x, const double* gx, double eps,
                       double* dc) {
    double* h = dalloc(I);
    double* q = dalloc(m);
    double* cs = dalloc(m);
    double* M = dalloc((int64_t)m * m);
    double* beta = dalloc(m);
    for (int32_t i = 0; i < I; ++i) {
        double s = 0.0;
        for (int32_t k = 0; k < m; ++k) s += x[(int64_t)i * m + k] * gx[(int64_t)i * m + k];
        h[i] = s;
    }
    for (int32_t k = 0; k < m; ++k) {
        double sq = 0.0, sc = 0.0, sh = 0.0;
        for (int32_t i = 0; i < I; ++i) {
            double xik = x[(int64_t)i * m + k];
            sq += xik * gx[(int64_t)i * m + k];
            sc += xik;
            sh += xik * h[i];
        }
        q[k] = sq;
        cs[k] = sc;
        beta[k] = sq - sh; /* right-hand side q - X^T h */
    }
    for (int32_t k = 0; k < m; ++k)
        for (int32_t l = 0; l < m; ++l) {
            double s = 0.0;
            for (int32_t i = 0; i < I; ++i) s += x[(int64_t)i * m + k] * x[(int64_t)i * m + l];
            M[(int64_t)k * m + l] = (k == l ? cs[k] : 0.0) - s;
        }
    /* gauge: drop the last column's equation and fix beta_{m-1} = 0 */
    int32_t n = m - 1;
    double* Ar = dalloc((int64_t)(n > 0 ? n : 1) * (n > 0 ? n : 1));
    for (int32_t k = 0; k < n; ++k)
        for (int32_t l = 0; l < n; ++l) Ar[(int64_t)k * n + l] = M[(int64_t)k * m + l];
    solve_spd(n, Ar, beta);
    beta[m - 1] = 0.0;
    for (int32_t i = 0; i < I; ++i) {
        double a = h[i];
        for (int32_t k = 0; k < m; ++k) a -= x[(int64_t)i * m + k] * beta[k];
        for (int32_t k = 0; k < m; ++k) {
            int64_t j = (int64_t)i * m + k;
            dc[j] = -(1.0 / eps) * x[j] * (gx[j] - a - beta[k]);
        }
    }
    free(h);
    free(q);
    free(cs);
    free(M);
    free(beta);
    free(Ar);
}

/* Reverse mode through the L-iteration Sinkhorn map of orc_sinkhorn: the chain-rule gradient of
 * Sec. 3 applied to the finite iteration itself rather than to its limit.
 * With g^(0) held constant, iteration l maps g^(l-1) -> f^(l) -> g^(l):
 *   P_ik = exp((f^l_i + g^{l-1}_k - c_ik)/eps)  (row-stochastic):  df_i/dg_k = -P_ik, df_i/dc_ik = P_ik
 *   Q_ik = exp((f^l_i + g^l_k - c_ik)/eps)/b_k (column-stochastic): dg_k/df_i = -Q_ik, dg_k/dc_ik = Q_ik
 * and the emitted policy is x_ik = softmax_k((g^{L-1}_k - c_ik)/eps). */
void orc_unrolled_grad(int32_t I, int32_t m, const double* c, const double* b, double eps,
                       int32_t L, const double* g0, const double* gx, double* dc) {
    double* gs = dalloc((int64_t)L * m); /* gs[l] = g^(l), l = 0..L-1 */
    double* fs = dalloc((int64_t)L * I); /* fs[l] = f^(l+1) */
    double* g = dalloc(m);
    double* buf = dalloc(I > m ? I : m);
    memcpy(g, g0, sizeof(double) * (size_t)m);
    for (int32_t l = 0; l < L; ++l) {
        memcpy(gs + (int64_t)l * m, g, sizeof(double) * (size_t)m);
        double* f = fs + (int64_t)l * I;
        for (int32_t i = 0; i < I; ++i) {
            for (int32_t k = 0; k < m; ++k) buf[k] = (g[k] - c[(int64_t)i * m + k]) / eps;
            f[i] = -eps * lse(buf, m);
        }
        for (int32_t k = 0; k < m; ++k) {
            for (int32_t i = 0; i < I; ++i) buf[i] = (f[i] - c[(int64_t)i * m + k]) / eps;
            g[k] = eps * log(b[k]) - eps * lse(buf, I);
        }
    }
    double* gbar = dalloc(m);
    double* gbar2 = dalloc(m);
    double* fbar = dalloc(I);
    for (int64_t j = 0; j < (int64_t)I * m; ++j) dc[j] = 0.0;
    /* output layer: x = softmax_k(z), z_ik = (g^{L-1}_k - c_ik)/eps */
    {
        const double* f = fs + (int64_t)(L - 1) * I;
        const double* gl = gs + (int64_t)(L - 1) * m;
        for (int32_t i = 0; i < I; ++i) {
            double h = 0.0;
            for (int32_t k = 0; k < m; ++k) {
                double x = exp((f[i] + gl[k] - c[(int64_t)i * m + k]) / eps);
                h += x * gx[(int64_t)i * m + k];
            }
            for (int32_t k = 0; k < m; ++k) {
                double x = exp((f[i] + gl[k] - c[(int64_t)i * m + k]) / eps);
                double zbar = x * (gx[(int64_t)i * m + k] - h);
                dc[(int64_t)i * m + k] -= zbar / eps;
                gbar[k] += zbar / eps;
            }
        }
    }
    for (int32_t l = L - 1; l >= 1; --l) {
        const double* f = fs + (int64_t)(l - 1) * I; /* f^(l) */
        const double* gl = gs + (int64_t)l * m;       /* g^(l) */
        const double* gp = gs + (int64_t)(l - 1) * m; /* g^(l-1) */
        for (int32_t i = 0; i < I; ++i) { /* through the column update */
            double s = 0.0;
            for (int32_t k = 0; k < m; ++k) {
                double Q = exp((f[i] + gl[k] - c[(int64_t)i * m + k]) / eps) / b[k];
                s -= Q * gbar[k];
                dc[(int64_t)i * m + k] += Q * gbar[k];
            }
            fbar[i] = s;
        }
        for (int32_t k = 0; k < m; ++k) gbar2[k] = 0.0;
        for (int32_t i = 0; i < I; ++i) { /* through the row update */
            for (int32_t k = 0; k < m; ++k) {
                double P = exp((f[i] + gp[k] - c[(int64_t)i * m + k]) / eps);
                gbar2[k] -= P * fbar[i];
                dc[(int64_t)i * m + k] += P * fbar[i];
            }
        }
        memcpy(gbar, gbar2, sizeof(double) * (size_t)m);
    }
    free(gs);
    free(fs);
    free(g);
    free(buf);
    free(gbar);
    free(gbar2);
    free(fbar);
}

/* Sec. 4.1: the ascent of Algorithm 1 is driven by PyTorch's Adam (Kingma & Ba).
 * Restated from the Adam paper with the bias-corrected denominator as torch documents it:
 *   m <- b1 m + (1-b1) g,  v <- b2 v + (1-b2) g^2,
 *   p <- p + (lr / (1-b1^t)) * m / (sqrt(v)/sqrt(1-b2^t) + eps)     (ascent: maximize=True). */
void orc_adam(int64_t n, double* p, double* mom1, double* mom2, const double* grad, int64_t t,
              double lr, double beta1, double beta2, double eps) {
    double bc1 = 1.0 - pow(beta1, (double)t);
    double bc2 = 1.0 - pow(beta2, (double)t);
    double step = lr / bc1, bc2s = sqrt(bc2);
    for (int64_t j = 0; j < n; ++j) {
        mom1[j] = beta1 * mom1[j] + (1.0 - beta1) * grad[j];
        mom2[j] = beta2 * mom2[j] + (1.0 - beta2) * grad[j] * grad[j];
        p[j] += step * mom1[j] / (sqrt(mom2[j]) / bc2s + eps);
    }
}

void orc_sgd(int64_t n, double* p, const double* grad, double lr) {
    for (int64_t j = 0; j < n; ++j) p[j] += lr * grad[j];
}

/* ---- Algorithm 1 engine ------------------------------------------------------------------- */

struct orc_ctx {
    orc_config cfg;
    int32_t U, I, K, m;
    double *b, *e;              /* m */
    double* r;                  /* U*I */
    int32_t have_r, have_e;
    int64_t nparam;             /* P1: U*I*m, P2: I */
    double *param, *mom1, *mom2;
    double *g, *g0, *gprev;     /* U*m: g^(L) (warm-start state), g^(0) and g^(L-1) of the last solve */
    double* X;                  /* U*I*m */
    double* imp;                /* I */
    double F;
    int64_t t;
    int32_t fresh;              /* policy X solved for the current parameters */
};

static int nthreads(const orc_ctx* ctx) {
    return ctx->cfg.n_threads > 0 ? ctx->cfg.n_threads : 1;
}

orc_ctx* orc_create(const orc_config* cfg) {
    if (!cfg || cfg->n_users < 1 || cfg->n_items < 1 || cfg->n_slots < 1 ||
        cfg->n_items < cfg->n_slots || cfg->sinkhorn_iters < 1 || !(cfg->epsilon > 0.0))
        return NULL;
    orc_ctx* ctx = (orc_ctx*)calloc(1, sizeof(orc_ctx));
    ctx->cfg = *cfg;
    ctx->U = cfg->n_users;
    ctx->I = cfg->n_items;
    ctx->K = cfg->n_slots;
    ctx->m = orc_num_cols(ctx->I, ctx->K);
    int64_t cells = (int64_t)ctx->U * ctx->I * ctx->m;
    ctx->nparam = cfg->param == ORC_PARAM_ITEM ? ctx->I : cells;
    ctx->b = dalloc(ctx->m);
    ctx->e = dalloc(ctx->m);
    ctx->r = dalloc((int64_t)ctx->U * ctx->I);
    ctx->param = dalloc(ctx->nparam);
    ctx->mom1 = dalloc(ctx->nparam);
    ctx->mom2 = dalloc(ctx->nparam);
    ctx->g = dalloc((int64_t)ctx->U * ctx->m);
    ctx->g0 = dalloc((int64_t)ctx->U * ctx->m);
    ctx->gprev = dalloc((int64_t)ctx->U * ctx->m);
    ctx->X = dalloc(cells);
    ctx->imp = dalloc(ctx->I);
    /* Algorithm 1 leaves the initial C unspecified; C = 0 (theta = 0) starts from the uniform
       ranking policy. */
    return ctx;
}

void orc_destroy(orc_ctx* ctx) {
    if (!ctx) return;
    free(ctx->b); free(ctx->e); free(ctx->r); free(ctx->param); free(ctx->mom1); free(ctx->mom2);
    free(ctx->g); free(ctx->g0); free(ctx->gprev); free(ctx->X); free(ctx->imp);
    free(ctx);
}

int32_t orc_set_relevance(orc_ctx* ctx, const double* r) {
    int64_t n = (int64_t)ctx->U * ctx->I;
    for (int64_t j = 0; j < n; ++j)
        if (!(r[j] >= 0.0) || !isfinite(r[j])) return 1;
    for (int32_t i = 0; i < ctx->I; ++i) { /* log Imp_i needs some positive relevance */
        int any = 0;
        for (int32_t u = 0; u < ctx->U; ++u) any |= r[(int64_t)u * ctx->I + i] > 0.0;
        if (!any) return 1;
    }
    memcpy(ctx->r, r, sizeof(double) * (size_t)n);
    ctx->have_r = 1;
    ctx->fresh = 0;
    return 0;
}

int32_t orc_set_exposure(orc_ctx* ctx, const double* e, int32_t K) {
    if (K != ctx->K) return 1;
    for (int32_t k = 0; k < K; ++k)
        if (!(e[k] > 0.0) || !isfinite(e[k])) return 1;
    orc_marginals(ctx->I, ctx->K, e, ctx->b, ctx->e);
    ctx->have_e = 1;
    ctx->fresh = 0;
    return 0;
}

int32_t orc_set_state(orc_ctx* ctx, const double* param, const double* mom1, const double* mom2,
                      const double* g, int64_t t) {
    size_t np = sizeof(double) * (size_t)ctx->nparam;
    if (param) memcpy(ctx->param, param, np);
    if (mom1) memcpy(ctx->mom1, mom1, np);
    if (mom2) memcpy(ctx->mom2, mom2, np);
    if (g) memcpy(ctx->g, g, sizeof(double) * (size_t)ctx->U * ctx->m);
    if (t < 0) return 1;
    ctx->t = t;
    ctx->fresh = 0;
    return 0;
}

int32_t orc_get_state(const orc_ctx* ctx, double* param, double* mom1, double* mom2, double* g,
                      int64_t* t) {
    size_t np = sizeof(double) * (size_t)ctx->nparam;
    if (param) memcpy(param, ctx->param, np);
    if (mom1) memcpy(mom1, ctx->mom1, np);
    if (mom2) memcpy(mom2, ctx->mom2, np);
    if (g) memcpy(g, ctx->g, sizeof(double) * (size_t)ctx->U * ctx->m);
    if (t) *t = ctx->t;
    return 0;
}

/* Cost matrix of consumer u into buf (P2) or a pointer into param (P1). */
static const double* consumer_cost(const orc_ctx* ctx, int32_t u, double* buf) {
    if (ctx->cfg.param == ORC_PARAM_ITEM) {
        orc_cost_item(ctx->I, ctx->m, ctx->r + (int64_t)u * ctx->I, ctx->e, ctx->param, buf);
        return buf;
    }
    return ctx->param + (int64_t)u * ctx->I * ctx->m;
}

/* Algorithm 1, parallel loop over consumers: X_u = X*_u(C_u) by Sinkhorn; then Eqs. (4)-(5). */
static void solve_all(orc_ctx* ctx) {
    const int32_t U = ctx->U, I = ctx->I, m = ctx->m;
#pragma omp parallel num_threads(nthreads(ctx))
    {
        double* buf = dalloc((int64_t)I * m);
#pragma omp for schedule(static)
        for (int32_t u = 0; u < U; ++u) {
            const double* c = consumer_cost(ctx, u, buf);
            double* g = ctx->g + (int64_t)u * m;
            if (!ctx->cfg.warm_start)
                for (int32_t k = 0; k < m; ++k) g[k] = 0.0;
            memcpy(ctx->g0 + (int64_t)u * m, g, sizeof(double) * (size_t)m);
            orc_sinkhorn(I, m, c, ctx->b, ctx->cfg.epsilon, ctx->cfg.sinkhorn_iters, g,
                         ctx->X + (int64_t)u * I * m, ctx->gprev + (int64_t)u * m);
        }
        free(buf);
    }
    /* Eq. (4): Imp_i = sum_u sum_{k < m-1} r(u,i) e(k) x_uik (dummy slot excluded) */
    for (int32_t i = 0; i < I; ++i) ctx->imp[i] = 0.0;
    for (int32_t u = 0; u < U; ++u)
        for (int32_t i = 0; i < I; ++i) {
            double s = 0.0;
            for (int32_t k = 0; k < ctx->K; ++k) s += ctx->e[k] * ctx->X[IDX3(u, i, k, I, m)];
            ctx->imp[i] += ctx->r[(int64_t)u * I + i] * s;
        }
    /* Eq. (5): F = sum_i log Imp_i */
    double F = 0.0;
    for (int32_t i = 0; i < I; ++i) F += log(ctx->imp[i]);
    ctx->F = F;
    ctx->fresh = 1;
}

/* Gradient of L = sum_i omega_i Imp_i at the current policy (omega_i = 1/Imp_i gives F, since
 * dF/dx_uik = r(u,i) e(k) / Imp_i). dparam: P1 dL/dC (U*I*m); P2 dL/dtheta (I). dr: U*I (nullable).
 * Returns ||dparam||_2^2. */
static double grad_all(orc_ctx* ctx, const double* omega_in, double* dparam, double* dr) {
    const int32_t U = ctx->U, I = ctx->I, m = ctx->m, K = ctx->K;
    const int p2 = ctx->cfg.param == ORC_PARAM_ITEM;
    double* omega = dalloc(I);
    for (int32_t i = 0; i < I; ++i) omega[i] = omega_in ? omega_in[i] : 1.0 / ctx->imp[i];
    double* dth_u = p2 ? dalloc((int64_t)U * I) : NULL; /* per-consumer theta contributions */
#pragma omp parallel num_threads(nthreads(ctx))
    {
        double* buf = dalloc((int64_t)I * m);
        double* gx = dalloc((int64_t)I * m);
        double* dcb = dalloc((int64_t)I * m);
#pragma omp for schedule(static)
        for (int32_t u = 0; u < U; ++u) {
            const double* x = ctx->X + (int64_t)u * I * m;
            const double* ru = ctx->r + (int64_t)u * I;
            for (int32_t i = 0; i < I; ++i)
                for (int32_t k = 0; k < m; ++k)
                    gx[(int64_t)i * m + k] = k < K ? omega[i] * ru[i] * ctx->e[k] : 0.0;
            double* dc = p2 ? dcb : dparam + (int64_t)u * I * m;
            if (ctx->cfg.grad_mode == ORC_GRAD_UNROLLED) {
                const double* c = consumer_cost(ctx, u, buf);
                orc_unrolled_grad(I, m, c, ctx->b, ctx->cfg.epsilon, ctx->cfg.sinkhorn_iters,
                                  ctx->g0 + (int64_t)u * m, gx, dc);
            } else {
                orc_implicit_grad(I, m, x, gx, ctx->cfg.epsilon, dc);
            }
            for (int32_t i = 0; i < I; ++i) {
                double w = p2 ? exp(ctx->param[i]) : 0.0;
                double rho = 0.0; /* sum_k e_k dL/dc_ik */
                double v = 0.0;   /* sum_{k<K} e_k x_ik */
                for (int32_t k = 0; k < m; ++k) rho += ctx->e[k] * dc[(int64_t)i * m + k];
                for (int32_t k = 0; k < K; ++k) v += ctx->e[k] * x[(int64_t)i * m + k];
                if (p2) dth_u[(int64_t)u * I + i] = -ru[i] * w * rho; /* dc/dtheta = -r e w */
                if (dr) dr[(int64_t)u * I + i] = omega[i] * v - (p2 ? w * rho : 0.0);
            }
        }
        free(buf);
        free(gx);
        free(dcb);
    }
    double n2 = 0.0;
    if (p2) {
        for (int32_t i = 0; i < I; ++i) dparam[i] = 0.0;
        for (int32_t u = 0; u < U; ++u)
            for (int32_t i = 0; i < I; ++i) dparam[i] += dth_u[(int64_t)u * I + i];
        for (int32_t i = 0; i < I; ++i) n2 += dparam[i] * dparam[i];
        free(dth_u);
    } else {
        for (int64_t j = 0; j < ctx->nparam; ++j) n2 += dparam[j] * dparam[j];
    }
    free(omega);
    return n2;
}

static int ready(const orc_ctx* ctx) { return ctx && ctx->have_r && ctx->have_e; }

/* One pass of Algorithm 1's loop body after the first solve: ascend C along grad F(X*(C)), then
 * re-solve every consumer. */
static double one_step(orc_ctx* ctx, double* dparam) {
    double n2 = grad_all(ctx, NULL, dparam, NULL);
    ctx->t += 1;
    if (ctx->cfg.optimizer == ORC_SGD)
        orc_sgd(ctx->nparam, ctx->param, dparam, ctx->cfg.lr);
    else
        orc_adam(ctx->nparam, ctx->param, ctx->mom1, ctx->mom2, dparam, ctx->t, ctx->cfg.lr,
                 ctx->cfg.beta1, ctx->cfg.beta2, ctx->cfg.adam_eps);
    solve_all(ctx);
    return sqrt(n2);
}

int32_t orc_step(orc_ctx* ctx, int32_t n, double* F_trace, double* gnorm_trace) {
    if (!ready(ctx) || n < 0) return 1;
    if (!ctx->fresh) solve_all(ctx);
    double* dparam = dalloc(ctx->nparam);
    for (int32_t s = 0; s < n; ++s) {
        double gn = one_step(ctx, dparam);
        if (F_trace) F_trace[s] = ctx->F;
        if (gnorm_trace) gnorm_trace[s] = gn;
    }
    free(dparam);
    return 0;
}

/* Algorithm 1 with threshold t on ||grad_C F||_2 (the gradient of Problem (8); the gradient with
 * respect to X never vanishes). The norm of a step's gradient is known once that step ran, so the
 * loop stops after the first step whose gradient norm is <= t. */
int32_t orc_solve(orc_ctx* ctx, double t, int32_t max_steps, int32_t* steps_done, double* F_out) {
    if (!ready(ctx) || max_steps < 0) return 1;
    if (!ctx->fresh) solve_all(ctx);
    double* dparam = dalloc(ctx->nparam);
    int32_t s = 0;
    while (s < max_steps) {
        double gn = one_step(ctx, dparam);
        ++s;
        if (gn <= t) break;
    }
    free(dparam);
    if (steps_done) *steps_done = s;
    if (F_out) *F_out = ctx->F;
    return 0;
}

int32_t orc_impacts(orc_ctx* ctx, double* imp, double* utility, double* F) {
    if (!ready(ctx)) return 1;
    if (!ctx->fresh) solve_all(ctx);
    double s = 0.0;
    for (int32_t i = 0; i < ctx->I; ++i) {
        if (imp) imp[i] = ctx->imp[i];
        s += ctx->imp[i];
    }
    if (utility) *utility = s / ctx->U; /* Sec. 4.1 user utility = sum_i Imp_i / |U| */
    if (F) *F = ctx->F;
    return 0;
}

int32_t orc_policy(orc_ctx* ctx, int32_t u0, int32_t n_u, double* x) {
    if (!ready(ctx) || u0 < 0 || n_u < 0 || u0 + n_u > ctx->U) return 1;
    if (!ctx->fresh) solve_all(ctx);
    memcpy(x, ctx->X + (int64_t)u0 * ctx->I * ctx->m,
           sizeof(double) * (size_t)n_u * ctx->I * ctx->m);
    return 0;
}

int32_t orc_grad(orc_ctx* ctx, const double* omega, double* dparam, double* dr) {
    if (!ready(ctx)) return 1;
    if (!ctx->fresh) solve_all(ctx);
    grad_all(ctx, omega, dparam, dr);
    return 0;
}

/* Sec. 4.1 metrics. Imp_i(X_j) = sum_u sum_{k<m-1} r(u,i) e(k) x_ujk is the impact item i would
 * get from item j's rankings; envy_i = max_j (Imp_i(X_j) - Imp_i(X_i)) (j = i allowed, so >= 0).
 * The uniform policy places every item at slot k with probability b_k/|I|. A change of more than 10% is
 * read as a strict ratio test against that policy's impact. */
int32_t orc_metrics(orc_ctx* ctx, double* utility, double* mean_envy, double* better_pct,
                    double* worse_pct) {
    if (!ready(ctx)) return 1;
    if (!ctx->fresh) solve_all(ctx);
    const int32_t U = ctx->U, I = ctx->I, m = ctx->m, K = ctx->K;
    double* V = dalloc((int64_t)U * I);
    for (int32_t u = 0; u < U; ++u)
        for (int32_t j = 0; j < I; ++j) {
            double s = 0.0;
            for (int32_t k = 0; k < K; ++k) s += ctx->e[k] * ctx->X[IDX3(u, j, k, I, m)];
            V[(int64_t)u * I + j] = s;
        }
    double env = 0.0;
#pragma omp parallel for num_threads(nthreads(ctx)) reduction(+ : env) schedule(static)
    for (int32_t i = 0; i < I; ++i) {
        double own = 0.0, best = -INFINITY;
        for (int32_t u = 0; u < U; ++u) own += ctx->r[(int64_t)u * I + i] * V[(int64_t)u * I + i];
        for (int32_t j = 0; j < I; ++j) {
            double s = 0.0;
            for (int32_t u = 0; u < U; ++u) s += ctx->r[(int64_t)u * I + i] * V[(int64_t)u * I + j];
            if (s - own > best) best = s - own;
        }
        env += best;
    }
    double esum = 0.0;
    for (int32_t k = 0; k < K; ++k) esum += ctx->e[k];
    int32_t nb = 0, nw = 0;
    double tot = 0.0;
    for (int32_t i = 0; i < I; ++i) {
        double ru = 0.0;
        for (int32_t u = 0; u < U; ++u) ru += ctx->r[(int64_t)u * I + i];
        double unif = ru * esum / I;
        if (ctx->imp[i] > 1.1 * unif) ++nb;
        if (ctx->imp[i] < 0.9 * unif) ++nw;
        tot += ctx->imp[i];
    }
    if (utility) *utility = tot / U;
    if (mean_envy) *mean_envy = env / I;
    if (better_pct) *better_pct = 100.0 * nb / I;
    if (worse_pct) *worse_pct = 100.0 * nw / I;
    free(V);
    return 0;
}

static int cmp_desc(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x < y) - (x > y);
}

/* Frank-Wolfe gap for Problem (6). F is concave in X and each X_u ranges over the transportation
 * polytope of Eqs. (1)-(3), so F* - F(X) <= max_Y <grad F(X), Y - X>. With dF/dx_uik =
 * r(u,i) e(k)/Imp_i and e non-increasing (dummy e = 0), the maximising Y_u places the K items with
 * the largest r(u,i)/Imp_i into slots 1..K in that order (rearrangement inequality). */
int32_t orc_certificate(orc_ctx* ctx, double* gap, double* col_residual) {
    if (!ready(ctx)) return 1;
    if (!ctx->fresh) solve_all(ctx);
    const int32_t U = ctx->U, I = ctx->I, m = ctx->m, K = ctx->K;
    double* rho = dalloc(I);
    double gsum = 0.0, res = 0.0;
    for (int32_t u = 0; u < U; ++u) {
        double lin = 0.0;
        for (int32_t i = 0; i < I; ++i) {
            rho[i] = ctx->r[(int64_t)u * I + i] / ctx->imp[i];
            for (int32_t k = 0; k < K; ++k) lin += rho[i] * ctx->e[k] * ctx->X[IDX3(u, i, k, I, m)];
        }
        qsort(rho, (size_t)I, sizeof(double), cmp_desc);
        double best = 0.0;
        for (int32_t k = 0; k < K; ++k) best += ctx->e[k] * rho[k];
        gsum += best - lin;
        for (int32_t k = 0; k < m; ++k) {
            double cs = 0.0;
            for (int32_t i = 0; i < I; ++i) cs += ctx->X[IDX3(u, i, k, I, m)];
            double d = fabs(cs - ctx->b[k]);
            if (d > res) res = d;
        }
    }
    if (gap) *gap = gsum;
    if (col_residual) *col_residual = res;
    free(rho);
    return 0;
}
