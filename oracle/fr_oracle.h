/*
 * fr_oracle.h -- plain FP64 CPU oracle for impact-based fair ranking solved by gradient
 * ascent over Sinkhorn solves (Uehara et al., "Fast solution to the fair ranking problem
 * using the Sinkhorn algorithm", arXiv 2406.10262).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load this library. It shares no source, header, table or helper with the
 * CUDA library; the two agree only on the meaning of the problem.
 *
 * Everything is double precision, row-major, plain loops. Notation follows the paper:
 *   U consumers, I items, K real ranking slots; m = K+1 columns when I > K (the last one is the
 *   dummy slot of Sec. 2 that absorbs the I-K unranked items), m = K when I == K.
 *   r[u*I+i]            relevance r(u,i)                                    (Sec. 2, Eq. 4)
 *   e[k], k < K         exposure e(k) of real slot k; the dummy slot has e = 0 (Eq. 4 sums k < m-1 only)
 *   X[(u*I+i)*m+k]      policy x_uik                                       (Sec. 2, Eqs. 1-3)
 *   C[(u*I+i)*m+k]      transport cost c_uik                                (Sec. 3, Problem (7))
 *
 * Parity status of each function is listed in the header comment of fr_oracle.c.
 */
#ifndef FR_ORACLE_H
#define FR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PARAM_FULL_C = 0, ORC_PARAM_ITEM = 1 };
enum { ORC_GRAD_IMPLICIT = 0, ORC_GRAD_UNROLLED = 1 };
enum { ORC_ADAM = 0, ORC_SGD = 1 };

typedef struct {
    int32_t n_users, n_items, n_slots; /* U, I, K */
    int32_t param;                     /* ORC_PARAM_FULL_C: free C (Problem (8)); ORC_PARAM_ITEM: c_uik = -r_ui e_k exp(theta_i) */
    double  epsilon;                   /* entropic regularisation of Problem (7) */
    int32_t sinkhorn_iters;            /* L >= 1 */
    int32_t warm_start;                /* 1: each solve starts from the previous solve's column potentials */
    int32_t grad_mode;                 /* ORC_GRAD_IMPLICIT | ORC_GRAD_UNROLLED */
    int32_t optimizer;                 /* ORC_ADAM | ORC_SGD */
    double  lr, beta1, beta2, adam_eps;
    int32_t n_threads;                 /* OpenMP threads over consumers (<=0: library default) */
} orc_config;

/* ---- stateless building blocks ------------------------------------------------------------ */

/* Column count m, column marginals b (length m) and padded exposure (length m, dummy = 0). */
int32_t orc_num_cols(int32_t I, int32_t K);
void orc_marginals(int32_t I, int32_t K, const double* e_in, double* b, double* e);

/* Log-domain Sinkhorn on one consumer (Problem (7)). g: in = g^(0), out = g^(L).
   x: out, the policy after the last row update (rows sum to exactly 1).
   gprev: out (nullable), g^(L-1), the column potentials that x was formed with. */
void orc_sinkhorn(int32_t I, int32_t m, const double* c, const double* b, double eps, int32_t L,
                  double* g, double* x, double* gprev);

/* Cost row block of one consumer under the per-item parametrisation:
   c_ik = -r_ui e_k exp(theta_i). */
void orc_cost_item(int32_t I, int32_t m, const double* r_u, const double* e, const double* theta,
                   double* c);

/* dF/dC of one consumer from the optimality conditions of Problem (7) at the emitted x
   (implicit differentiation). gx = dF/dx. */
void orc_implicit_grad(int32_t I, int32_t m, const double* x, const double* gx, double eps,
                       double* dc);

/* dF/dC of one consumer by reverse mode through the L-iteration Sinkhorn map started from g0
   (g0 held constant). gx = dF/dx for the emitted x. */
void orc_unrolled_grad(int32_t I, int32_t m, const double* c, const double* b, double eps,
                       int32_t L, const double* g0, const double* gx, double* dc);

/* Adam exactly as torch.optim.Adam(maximize=True) documents it, one step (t is the new step
   count, >= 1); SGD ascent. grad is the ascent direction dF/dparam. */
void orc_adam(int64_t n, double* p, double* mom1, double* mom2, const double* grad, int64_t t,
              double lr, double beta1, double beta2, double eps);
void orc_sgd(int64_t n, double* p, const double* grad, double lr);

/* ---- engine: Algorithm 1 with state ------------------------------------------------------ */

typedef struct orc_ctx orc_ctx;

orc_ctx* orc_create(const orc_config* cfg);
void     orc_destroy(orc_ctx* ctx);
/* Returns 0 on success, nonzero on invalid input (negative/non-finite r, an item with no positive
   relevance, non-positive exposure, K mismatch). */
int32_t  orc_set_relevance(orc_ctx* ctx, const double* r);
int32_t  orc_set_exposure(orc_ctx* ctx, const double* e, int32_t K);
/* Optimiser state: param (P1: U*I*m, P2: I), Adam moments (same shapes), column potentials g
   (U*m) and step count t. Setting state marks the policy as stale (the next step re-solves). */
int32_t  orc_set_state(orc_ctx* ctx, const double* param, const double* mom1, const double* mom2,
                       const double* g, int64_t t);
int32_t  orc_get_state(const orc_ctx* ctx, double* param, double* mom1, double* mom2, double* g,
                       int64_t* t);
/* n ascent steps. If the policy is stale, first solves Sinkhorn for the current parameters.
   Each step: gradient at the current policy, optimiser update, Sinkhorn for the new parameters,
   impacts and F. F_trace (nullable, length n) receives F after each step; gnorm_trace (nullable)
   the 2-norm of the gradient each step used. */
int32_t  orc_step(orc_ctx* ctx, int32_t n, double* F_trace, double* gnorm_trace);
/* Algorithm 1 with threshold t: steps until a step's gradient norm is <= t (that step's update is
   still applied), or max_steps. */
int32_t  orc_solve(orc_ctx* ctx, double t, int32_t max_steps, int32_t* steps_done, double* F_out);
/* Solves Sinkhorn for the current parameters if stale and reports impacts (I), utility and F. */
int32_t  orc_impacts(orc_ctx* ctx, double* imp, double* utility, double* F);
int32_t  orc_policy(orc_ctx* ctx, int32_t u0, int32_t n_u, double* x);
/* Gradient of L = sum_i omega_i Imp_i (omega nullable: omega_i = 1/Imp_i, i.e. L = F) at the current
   policy, in the configured grad_mode: dparam (P1: U*I*m, P2: I) and, for P2, dr (U*I, nullable). */
int32_t  orc_grad(orc_ctx* ctx, const double* omega, double* dparam, double* dr);
/* Evaluation metrics of Sec. 4.1 at the current policy: user utility, mean max envy, percentage of
   items better off / worse off by more than 10% relative to the uniform policy. */
int32_t  orc_metrics(orc_ctx* ctx, double* utility, double* mean_envy, double* better_pct,
                     double* worse_pct);
/* Frank-Wolfe duality gap of the current policy for Problem (6): an upper bound on F* - F when the
   policy is feasible and e is non-increasing. Also returns the max column-marginal residual. */
int32_t  orc_certificate(orc_ctx* ctx, double* gap, double* col_residual);

#ifdef __cplusplus
}
#endif
#endif
