// fr_api.cu -- the extern "C" entry points of libfairrank (include/fairrank.h).
//
// Host side of Algorithm 1: argument checking, device memory, stream ordering and the CUDA graphs
// that replay chunks of ascent steps. Every step of the method itself runs in the kernels of
// fr_p1.cu (free costs: Sinkhorn, impacts, gradient, Adam), fr_p2*.cu (per-item variables) and
// fr_common.cu (cross-consumer reduction).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "fairrank.h"
#include "fr_internal.h"

using namespace fr;

namespace {
thread_local std::string g_create_error;
constexpr int kChunk = 16;  // ascent steps per captured graph
}

struct fr_ctx {
    fr_config cfg;
    bool p2 = false;  // per-item parametrisation
    int U = 0, I = 0, K = 0, nc = 0, ld = 0, G = 0, nblk = 0;
    int device = 0;
    cudaStream_t user = nullptr;  // caller's stream (may be the legacy default stream)
    cudaStream_t s = nullptr;     // library stream (non-blocking), joined to `user` per call
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    P1Variant var{};
    P2Variant var2{};
    P1AdjVariant var1a{};  // free costs, unrolled gradient
    float* g0 = nullptr;   // free costs, unrolled gradient: [U][nc] starting potentials of the last solve
    float *gall = nullptr, *csall = nullptr;  // free costs, ce == 1: [U][L][nc] g' and cs per iteration
    int r_bf16 = 0;
    float emax = 0.f;
    double esum = 0.0;  // sum of the K real exposures (uniform-policy impacts of the metrics)
    // free costs: C, Adam moments [U][nc][ld]; per-item: theta, moments, w = exp(theta) [ld]
    float *C = nullptr, *m1 = nullptr, *m2 = nullptr;
    float *theta = nullptr, *tm1 = nullptr, *tm2 = nullptr, *w = nullptr, *gpart = nullptr;
    // unrolled differentiation (per-item): checkpoints g^(j ce) of the last sweep [U][nck][nc],
    // and the grid of the adjoint kernel (its dL/dtheta partials fill gpart[Gg][ld])
    bool unrolled = false;
    float* ck = nullptr;
    float* csk = nullptr;  // with ce == 1: the column sums of every iteration [U][L][nc]
    int ce = 0, nck = 0, Gg = 0;
    double *ad_blk = nullptr, *gn2_one = nullptr;
    float *gL = nullptr, *gP = nullptr, *e = nullptr, *invb = nullptr, *omega = nullptr,
          *part = nullptr;
    void* r = nullptr;  // [U][ld] float or bfloat16
    float* tmp = nullptr;  // staging for host transfers
    size_t tmp_bytes = 0;
    double *gn2_part = nullptr, *imp = nullptr, *blk = nullptr, *F_hist = nullptr, *gn_hist = nullptr;
    int hist_cap = 0;
    int hist_n = 0;  // steps recorded in F_hist / gn_hist by the last fr_step or fr_solve
    DevState* st = nullptr;
    DevState* st_host = nullptr;  // pinned
    int* flags = nullptr;
    bool have_r = false, have_e = false, fresh = false;
    cudaGraphExec_t chunk_exec = nullptr;
    cudaGraphExec_t solve_exec = nullptr;  // fr_solve: device-side while loop over step chunks
    int* solve_ctl = nullptr;              // [2] body iterations, cap
    int64_t launches = 0;
    std::string err;
};

namespace {

fr_status fail(fr_ctx* c, fr_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c)
        c->err = buf;
    else
        g_create_error = buf;
    return st;
}

// A failing runtime call returns its status with the message; its (non-sticky) error is also
// cleared from the runtime's last-error state, so that it cannot surface in a later call's checks.
#define CU(call)                                                                             \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            cudaGetLastError();                                                              \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? FR_ENOMEM : FR_ECUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                      \
        }                                                                                    \
    } while (0)

// Orders the library stream after the caller's stream (call entry) and back (call exit).
struct Join {
    fr_ctx* c;
    explicit Join(fr_ctx* ctx) : c(ctx) {
        cudaEventRecord(c->ev_in, c->user);
        cudaStreamWaitEvent(c->s, c->ev_in, 0);
    }
    ~Join() {
        cudaEventRecord(c->ev_out, c->s);
        cudaStreamWaitEvent(c->user, c->ev_out, 0);
    }
};

P1Args p1_args(fr_ctx* c) {
    P1Args a{};
    a.U = c->U; a.I = c->I; a.K = c->K; a.nc = c->nc; a.ld = c->ld;
    a.L = c->cfg.sinkhorn_iters; a.G = c->G;
    a.C = c->C; a.m1 = c->m1; a.m2 = c->m2; a.gL = c->gL; a.gP = c->gP;
    a.r = static_cast<const float*>(c->r); a.e = c->e; a.invb = c->invb; a.omega = c->omega;
    a.part = c->part; a.gn2_part = c->gn2_part; a.st = c->st;
    a.inv_eps_ln2 = (float)(1.0 / (c->cfg.epsilon * std::log(2.0)));
    a.inv_eps = (float)(1.0 / c->cfg.epsilon);
    a.lr = (float)c->cfg.lr; a.beta1 = (float)c->cfg.beta1; a.beta2 = (float)c->cfg.beta2;
    a.adam_eps = (float)c->cfg.adam_eps;
    a.optimizer = c->cfg.optimizer == FR_SGD ? 1 : 0;
    a.warm = c->cfg.warm_start ? 1 : 0;
    a.max_polls = polls_of(c->cfg.max_wait_polls);
    a.g0 = c->g0;
    a.gall = c->gall;
    a.csall = c->csall;
    a.ce = c->ce;
    a.nck = c->nck;
    return a;
}

P2Args p2_args(fr_ctx* c, float* part) {
    P2Args a{};
    a.U = c->U; a.I = c->I; a.K = c->K; a.nc = c->nc; a.ld = c->ld;
    a.L = c->cfg.sinkhorn_iters; a.G = c->G;
    a.r = c->r; a.r_bf16 = c->r_bf16; a.w = c->w; a.e = c->e; a.invb = c->invb;
    a.emax = c->emax; a.gL = c->gL; a.gP = c->gP; a.part = part; a.omega = c->omega;
    a.dr = nullptr; a.st = c->st;
    a.inv_eps_ln2 = (float)(1.0 / (c->cfg.epsilon * std::log(2.0)));
    a.inv_eps = (float)(1.0 / c->cfg.epsilon);
    a.warm = c->cfg.warm_start ? 1 : 0;
    a.ck = c->ck; a.ce = c->ce; a.nck = c->nck; a.csk = c->csk;
    a.max_polls = polls_of(c->cfg.max_wait_polls);
    return a;
}

// Gradient of sum_i omega_i Imp_i onto the per-CTA dL/dtheta partials gpart: implicit (Sec. 3
// optimality conditions) or through the unrolled iterations (adjoint kernel).
cudaError_t launch_p2_grad(fr_ctx* c, P2Args a) {
    a.part = c->gpart;
    a.G = c->Gg;
    return c->unrolled ? p2_launch_adj(c->var2, a, c->s) : p2_launch_grad(c->var2, a, c->s);
}

P2AdamArgs adam_args(fr_ctx* c, int apply, float* dtheta_out) {
    P2AdamArgs a{};
    a.I = c->I; a.ld = c->ld; a.G = c->Gg; a.part = c->gpart;
    a.theta = c->theta; a.m1 = c->tm1; a.m2 = c->tm2; a.w = c->w; a.dtheta_out = dtheta_out;
    a.gn2_out = c->gn2_one; a.blk = c->ad_blk; a.st = c->st;
    a.lr = (float)c->cfg.lr; a.beta1 = (float)c->cfg.beta1; a.beta2 = (float)c->cfg.beta2;
    a.adam_eps = (float)c->cfg.adam_eps;
    a.optimizer = c->cfg.optimizer == FR_SGD ? 1 : 0;
    a.apply = apply;
    return a;
}

ReduceArgs red_args(fr_ctx* c, int after_update) {
    ReduceArgs a{};
    a.I = c->I; a.ld = c->ld; a.G = c->G; a.U = c->U;
    a.part = c->part; a.imp = c->imp; a.omega = c->omega;
    a.blk = c->blk; a.st = c->st; a.F_hist = c->F_hist; a.gn_hist = c->gn_hist;
    a.hist_cap = c->hist_cap; a.after_update = after_update;
    if (c->p2) {
        a.gn2_part = c->gn2_one;
        a.Ggn = 1;
    } else {
        a.gn2_part = c->gn2_part;
        a.Ggn = c->unrolled ? c->Gg : c->G;  // the adjoint kernel's grid writes the norm partials
    }
    return a;
}

// Sinkhorn for every consumer at the current parameters, then impacts and F.
fr_status launch_solve(fr_ctx* ctx) {
    if (ctx->p2)
        CU(p2_launch_sweep(ctx->var2, p2_args(ctx, ctx->part), ctx->s));
    else
        CU(p1_launch(ctx->var, MODE_SWEEP, p1_args(ctx), ctx->s));
    CU(reduce_launch(red_args(ctx, 0), ctx->s));
    ctx->launches += 2;
    return FR_OK;
}

// One ascent step of Algorithm 1: gradient at the current policy, update, Sinkhorn, impacts.
fr_status launch_one_step(fr_ctx* ctx) {
    if (ctx->p2) {
        CU(launch_p2_grad(ctx, p2_args(ctx, ctx->gpart)));
        CU(p2_launch_adam(adam_args(ctx, 1, nullptr), ctx->s));
        CU(p2_launch_sweep(ctx->var2, p2_args(ctx, ctx->part), ctx->s));
        ctx->launches += 3;
    } else if (ctx->unrolled) {  // adjoint + optimiser, then Sinkhorn on the new costs
        CU(p1_launch_adj(ctx->var1a, 1, p1_args(ctx), ctx->Gg, ctx->s));
        CU(p1_launch(ctx->var, MODE_SWEEP, p1_args(ctx), ctx->s));
        ctx->launches += 2;
    } else {
        CU(p1_launch(ctx->var, MODE_UPDATE_SWEEP, p1_args(ctx), ctx->s));
        ctx->launches += 1;
    }
    CU(reduce_launch(red_args(ctx, 1), ctx->s));
    ctx->launches += 1;
    return FR_OK;
}

int kernels_per_step(const fr_ctx* c) { return c->p2 ? 4 : c->unrolled ? 3 : 2; }

fr_status ensure_fresh(fr_ctx* ctx) {
    if (!ctx->have_r || !ctx->have_e)
        return fail(ctx, FR_ESTATE, "set relevance and exposure first");
    if (ctx->fresh) return FR_OK;
    fr_status st = launch_solve(ctx);
    if (st != FR_OK) return st;
    ctx->fresh = true;
    return FR_OK;
}

fr_status ensure_hist(fr_ctx* ctx, int n) {
    if (n <= ctx->hist_cap) return FR_OK;
    int cap = ctx->hist_cap > 0 ? ctx->hist_cap : 64;
    while (cap < n) cap *= 2;
    CU(cudaStreamSynchronize(ctx->s));
    cudaFree(ctx->F_hist);
    cudaFree(ctx->gn_hist);
    ctx->F_hist = ctx->gn_hist = nullptr;
    CU(cudaMalloc(&ctx->F_hist, sizeof(double) * cap));
    CU(cudaMalloc(&ctx->gn_hist, sizeof(double) * cap));
    ctx->hist_cap = cap;
    if (ctx->chunk_exec) {  // kernel arguments changed: recapture
        cudaGraphExecDestroy(ctx->chunk_exec);
        ctx->chunk_exec = nullptr;
    }
    if (ctx->solve_exec) {
        cudaGraphExecDestroy(ctx->solve_exec);
        ctx->solve_exec = nullptr;
    }
    return FR_OK;
}

// fr_solve's graph: a conditional while node whose body is kChunk ascent steps followed by
// solve_cond_kernel, which keeps the loop running until the reduction raises the stop flag (the
// gradient-norm threshold or the step cap) -- no host round trip per chunk.
fr_status ensure_solve_graph(fr_ctx* ctx) {
    if (ctx->solve_exec) return FR_OK;
    if (!ctx->solve_ctl) CU(cudaMalloc(&ctx->solve_ctl, sizeof(int) * 2));
    cudaGraph_t g = nullptr;
    CU(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams p{};
    cudaGraphNode_t node;
    if (e == cudaSuccess) {
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &p);
    }
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        CU(e);
    }
    cudaGraph_t body = p.conditional.phGraph_out[0];
    const int64_t before = ctx->launches;
    CU(cudaStreamBeginCaptureToGraph(ctx->s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    fr_status st = FR_OK;
    for (int j = 0; j < kChunk && st == FR_OK; ++j) st = launch_one_step(ctx);
    if (st == FR_OK) st = launch_solve_cond(ctx->st, ctx->solve_ctl, h, ctx->s) == cudaSuccess ? FR_OK : FR_ECUDA;
    cudaGraph_t captured = nullptr;
    e = cudaStreamEndCapture(ctx->s, &captured);
    ctx->launches = before;  // captured, not launched
    if (st != FR_OK || e != cudaSuccess) {
        cudaGraphDestroy(g);
        if (st != FR_OK) return fail(ctx, st, "capturing the solve loop failed");
        CU(e);
    }
    e = cudaGraphInstantiate(&ctx->solve_exec, g, 0);
    cudaGraphDestroy(g);
    CU(e);
    return FR_OK;
}

fr_status ensure_graph(fr_ctx* ctx) {
    if (ctx->chunk_exec) return FR_OK;
    cudaGraph_t g = nullptr;
    CU(cudaStreamBeginCapture(ctx->s, cudaStreamCaptureModeThreadLocal));
    const int64_t before = ctx->launches;
    for (int j = 0; j < kChunk; ++j) {
        fr_status st = launch_one_step(ctx);
        if (st != FR_OK) {
            cudaStreamEndCapture(ctx->s, &g);
            if (g) cudaGraphDestroy(g);
            ctx->launches = before;
            return st;
        }
    }
    ctx->launches = before;  // captured, not launched
    CU(cudaStreamEndCapture(ctx->s, &g));
    cudaError_t e = cudaGraphInstantiate(&ctx->chunk_exec, g, 0);
    cudaGraphDestroy(g);
    CU(e);
    return FR_OK;
}

// Writes selected host-side fields of the device step state.
fr_status set_run_state(fr_ctx* ctx, double thresh, int max_steps = 0) {
    DevState* h = ctx->st_host;
    CU(cudaMemcpyAsync(h, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    h->hist_idx = 0;
    h->stop = 0;
    h->steps_done = 0;
    h->thresh = thresh;
    h->max_steps = max_steps;
    CU(cudaMemcpyAsync(ctx->st, h, sizeof(DevState), cudaMemcpyHostToDevice, ctx->s));
    return FR_OK;
}

fr_status read_state(fr_ctx* ctx) {
    CU(cudaMemcpyAsync(ctx->st_host, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    if (ctx->st_host->err & 4)
        return fail(ctx, FR_ETIMEOUT, "a bounded wait for a staged bulk copy expired");
    if (ctx->st_host->err)
        return fail(ctx, FR_ENUMERIC, "non-finite or non-positive impact (flags %d)",
                    ctx->st_host->err);
    return FR_OK;
}

// Runs n steps: whole chunks by graph replay, the remainder by direct launches.
fr_status run_steps(fr_ctx* ctx, int n) {
    int done = 0;
    if (n >= kChunk) {
        fr_status st = ensure_graph(ctx);
        if (st != FR_OK) return st;
    }
    while (n - done >= kChunk) {
        CU(cudaGraphLaunch(ctx->chunk_exec, ctx->s));
        ctx->launches += (int64_t)kernels_per_step(ctx) * kChunk;
        done += kChunk;
    }
    for (; done < n; ++done) {
        fr_status st = launch_one_step(ctx);
        if (st != FR_OK) return st;
    }
    return FR_OK;
}

fr_status ensure_tmp(fr_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->tmp_bytes) return FR_OK;
    CU(cudaStreamSynchronize(ctx->s));
    cudaFree(ctx->tmp);
    ctx->tmp = nullptr;
    ctx->tmp_bytes = 0;
    CU(cudaMalloc(&ctx->tmp, bytes));
    ctx->tmp_bytes = bytes;
    return FR_OK;
}

void free_all(fr_ctx* c) {
    if (c->chunk_exec) cudaGraphExecDestroy(c->chunk_exec);
    if (c->solve_exec) cudaGraphExecDestroy(c->solve_exec);
    cudaFree(c->solve_ctl);
    float* fs[] = {c->C, c->m1, c->m2, c->theta, c->tm1, c->tm2, c->w, c->gpart, c->gL, c->gP,
                   c->e, c->invb, c->omega, c->part, c->tmp, c->ck, c->csk, c->g0, c->gall,
                   c->csall};
    for (float* p : fs) cudaFree(p);
    double* ds[] = {c->gn2_part, c->imp, c->blk, c->F_hist, c->gn_hist, c->ad_blk, c->gn2_one};
    for (double* p : ds) cudaFree(p);
    cudaFree(c->r);
    cudaFree(c->st);
    cudaFree(c->flags);
    if (c->st_host) cudaFreeHost(c->st_host);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->s) cudaStreamDestroy(c->s);
}

size_t nparam(const fr_ctx* c) {  // public parameter count
    return c->p2 ? (size_t)c->I : (size_t)c->U * c->I * c->nc;
}

fr_status zero_state(fr_ctx* ctx) {
    if (ctx->p2) {
        CU(cudaMemsetAsync(ctx->theta, 0, sizeof(float) * ctx->ld, ctx->s));
        CU(cudaMemsetAsync(ctx->tm1, 0, sizeof(float) * ctx->ld, ctx->s));
        CU(cudaMemsetAsync(ctx->tm2, 0, sizeof(float) * ctx->ld, ctx->s));
        CU(launch_exp_theta(ctx->theta, ctx->w, ctx->I, ctx->ld, ctx->s));
        ctx->launches += 1;
    } else {
        const size_t cells = (size_t)ctx->U * ctx->nc * ctx->ld;
        CU(cudaMemsetAsync(ctx->C, 0, sizeof(float) * cells, ctx->s));
        CU(cudaMemsetAsync(ctx->m1, 0, sizeof(float) * cells, ctx->s));
        CU(cudaMemsetAsync(ctx->m2, 0, sizeof(float) * cells, ctx->s));
    }
    CU(cudaMemsetAsync(ctx->gL, 0, sizeof(float) * ctx->U * ctx->nc, ctx->s));
    CU(cudaMemsetAsync(ctx->gP, 0, sizeof(float) * ctx->U * ctx->nc, ctx->s));
    DevState z{};
    z.thresh = -1.0;
    *ctx->st_host = z;
    CU(cudaMemcpyAsync(ctx->st, ctx->st_host, sizeof(DevState), cudaMemcpyHostToDevice, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    ctx->fresh = false;
    return FR_OK;
}

}  // namespace

namespace fr {
// Message slot of fr_last_error(NULL) for entry points that take no context.
void set_thread_error(const char* msg) { g_create_error = msg; }
}  // namespace fr

extern "C" {

void fr_config_default(fr_config* cfg, int32_t n_users, int32_t n_items, int32_t n_slots,
                       int32_t param) {
    std::memset(cfg, 0, sizeof *cfg);
    cfg->n_users = n_users;
    cfg->n_items = n_items;
    cfg->n_slots = n_slots;
    cfg->param = param;
    cfg->epsilon = 1.0;
    cfg->sinkhorn_iters = 50;
    cfg->warm_start = 1;
    cfg->grad_mode = FR_GRAD_IMPLICIT;
    cfg->ckpt_every = 10;
    cfg->optimizer = FR_ADAM;
    cfg->lr = param == FR_PARAM_ITEM ? 0.05 : 0.1;
    cfg->beta1 = 0.9;
    cfg->beta2 = 0.999;
    cfg->adam_eps = 1e-8;
    cfg->rel_dtype = FR_F32;
}

int32_t fr_num_cols(int32_t n_items, int32_t n_slots) {
    return n_items > n_slots ? n_slots + 1 : n_slots;
}

fr_status fr_create(const fr_config* cfg, void* stream, fr_ctx** out) {
    NvtxRange nvtx_range("fr_create");
    fr_ctx* ctx = nullptr;
    if (!out) return fail(nullptr, FR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfg) return fail(nullptr, FR_EINVAL, "cfg is NULL");
    const fr_config& c = *cfg;
    if (c.n_users < 1 || c.n_items < 1 || c.n_slots < 1 || c.n_slots > c.n_items)
        return fail(nullptr, FR_EINVAL, "need n_users >= 1 and 1 <= n_slots <= n_items (got %d, %d, %d)",
                    c.n_users, c.n_items, c.n_slots);
    if (!(c.epsilon > 0.0) || !std::isfinite(c.epsilon))
        return fail(nullptr, FR_EINVAL, "epsilon must be positive and finite");
    if (c.sinkhorn_iters < 1) return fail(nullptr, FR_EINVAL, "sinkhorn_iters must be >= 1");
    if (!(c.lr > 0.0) || !(c.beta1 >= 0.0 && c.beta1 < 1.0) || !(c.beta2 >= 0.0 && c.beta2 < 1.0) ||
        !(c.adam_eps >= 0.0))
        return fail(nullptr, FR_EINVAL, "invalid optimiser hyper-parameters");
    if (c.optimizer != FR_ADAM && c.optimizer != FR_SGD)
        return fail(nullptr, FR_EINVAL, "unknown optimizer %d", c.optimizer);
    if (c.param != FR_PARAM_FULL_C && c.param != FR_PARAM_ITEM)
        return fail(nullptr, FR_EINVAL, "unknown param %d", c.param);
    if (c.grad_mode != FR_GRAD_IMPLICIT && c.grad_mode != FR_GRAD_UNROLLED)
        return fail(nullptr, FR_EINVAL, "unknown grad_mode %d", c.grad_mode);
    if (c.grad_mode == FR_GRAD_UNROLLED && c.ckpt_every < 1)
        return fail(nullptr, FR_EINVAL, "ckpt_every must be >= 1 (got %d)", c.ckpt_every);
    if (c.rel_dtype != FR_F32 && c.rel_dtype != FR_BF16)
        return fail(nullptr, FR_EINVAL, "rel_dtype must be FR_F32 or FR_BF16");
    if (c.param == FR_PARAM_FULL_C && c.rel_dtype != FR_F32)
        return fail(nullptr, FR_EUNSUPPORTED, "FR_PARAM_FULL_C stores relevance in FP32");
    for (int j = 0; j < 6; ++j)
        if (c.reserved[j]) return fail(nullptr, FR_EINVAL, "reserved fields must be zero");
    if (c.max_wait_polls < -1)
        return fail(nullptr, FR_EINVAL, "max_wait_polls must be >= -1 (got %d)", c.max_wait_polls);

    const int nc = fr_num_cols(c.n_items, c.n_slots);
    const bool p2 = c.param == FR_PARAM_ITEM;
    P1Variant var{};
    P2Variant var2{};
    P1AdjVariant var1a{};
    if (p2) {
        if (!p2_select(nc, c.n_items, &var2))
            return fail(nullptr, FR_EUNSUPPORTED,
                        "FR_PARAM_ITEM needs n_cols <= 32 and n_items <= 12288 (4096 unless "
                        "n_cols is 6, 11 or 21); got n_cols %d, n_items %d",
                        nc, c.n_items);
        if (c.grad_mode == FR_GRAD_UNROLLED && !p2_select_adj(nc, c.n_items, &var2))
            return fail(nullptr, FR_EUNSUPPORTED,
                        "unrolled differentiation needs n_items <= 6144 (2048 unless n_cols is 6, "
                        "11 or 21) and n_cols <= 32; got n_cols %d, n_items %d",
                        nc, c.n_items);
    } else if (!p1_select(nc, c.n_items, &var)) {
        return fail(nullptr, FR_EUNSUPPORTED,
                    "FR_PARAM_FULL_C needs n_cols <= 64 and n_items <= 512 * rows per thread "
                    "(2048 for n_cols <= 16, 1024 for <= 32, 512 for <= 64); got n_cols %d, n_items %d",
                    nc, c.n_items);
    } else if (c.grad_mode == FR_GRAD_UNROLLED && !p1_select_adj(nc, c.n_items, &var1a)) {
        return fail(nullptr, FR_EUNSUPPORTED,
                    "unrolled differentiation of FR_PARAM_FULL_C needs n_cols <= 32 and n_items <= "
                    "1024 (n_cols <= 16) or 512 (n_cols up to 32); got n_cols %d, n_items %d",
                    nc, c.n_items);
    }
    ctx = new fr_ctx();
    ctx->cfg = c;
    ctx->p2 = p2;
    ctx->U = c.n_users;
    ctx->I = c.n_items;
    ctx->K = c.n_slots;
    ctx->nc = nc;
    ctx->ld = (c.n_items + 7) / 8 * 8;
    ctx->var = var;
    ctx->var2 = var2;
    ctx->var1a = var1a;
    ctx->r_bf16 = c.rel_dtype == FR_BF16 ? 1 : 0;
    ctx->user = (cudaStream_t)stream;
    ctx->unrolled = c.grad_mode == FR_GRAD_UNROLLED;
    if (ctx->unrolled) {
        ctx->ce = std::min(c.ckpt_every, c.sinkhorn_iters);
        ctx->nck = (c.sinkhorn_iters + ctx->ce - 1) / ctx->ce;
    }
    auto bail = [&](fr_status st) {
        g_create_error = ctx->err;
        free_all(ctx);
        delete ctx;
        cudaGetLastError();  // a failed allocation must not surface in the next call's checks
        return st;
    };
#define CUC(call)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bail(fail(ctx, e_ == cudaErrorMemoryAllocation ? FR_ENOMEM : FR_ECUDA,     \
                             "%s: %s", #call, cudaGetErrorString(e_)));                       \
    } while (0)
    CUC(cudaGetDevice(&ctx->device));
    CUC(cudaStreamCreateWithFlags(&ctx->s, cudaStreamNonBlocking));
    CUC(cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming));
    CUC(cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming));

    // shared memory and occupancy fix the persistent grid G
    int max_optin = 0, sms = 0, occ = 0;
    CUC(cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
    CUC(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    auto set_smem = [&](const void* fn, size_t b) -> fr_status {
        if (b > (size_t)max_optin)
            return fail(ctx, FR_EUNSUPPORTED,
                        "shared memory %zu B exceeds the device limit %d B for this shape", b,
                        max_optin);
        cudaError_t e = raise_smem_limit(fn, b);
        if (e != cudaSuccess) return fail(ctx, FR_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
        return FR_OK;
    };
    if (p2) {
        const int esz = ctx->r_bf16 ? 2 : 4;
        const size_t bs = p2_sweep_smem(var2, nc, ctx->ld, esz);
        const size_t bg = p2_grad_smem(var2, nc, ctx->ld, esz);
        fr_status st = set_smem(var2.sweep, bs);
        if (st == FR_OK) st = set_smem(var2.grad, bg);
        if (st != FR_OK) return bail(st);
        int o1 = 0, o2 = 0;
        CUC(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, var2.sweep, var2.threads, bs));
        CUC(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, var2.grad, var2.threads, bg));
        occ = std::min(o1, o2);
        int og = o2;
        if (ctx->unrolled) {
            const size_t ba = p2_adj_smem(var2, nc, ctx->ld, esz, ctx->ce);
            if ((st = set_smem(var2.adj, ba)) != FR_OK) return bail(st);
            CUC(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&og, var2.adj, var2.adj_threads, ba));
            if (og < 1) return bail(fail(ctx, FR_EUNSUPPORTED, "adjoint kernel does not fit on an SM"));
        }
        ctx->Gg = std::min(ctx->U, std::max(og, 1) * sms);
    } else {
        for (int m = 0; m < 3; ++m) {
            fr_status st = set_smem(var.fn[m], p1_smem_bytes(var, m, nc, ctx->ld));
            if (st != FR_OK) return bail(st);
        }
        if (var.fn_rec) {
            fr_status st = set_smem(var.fn_rec, p1_smem_bytes(var, MODE_SWEEP, nc, ctx->ld));
            if (st != FR_OK) return bail(st);
        }
        CUC(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &occ, var.fn[MODE_UPDATE_SWEEP], var.threads,
            p1_smem_bytes(var, MODE_UPDATE_SWEEP, nc, ctx->ld)));
        if (ctx->unrolled) {
            const size_t ba = p1_adj_smem(var1a, nc, ctx->ld, ctx->ce, ctx->nck);
            int og = 0;
            for (int m = 0; m < 2; ++m) {
                fr_status st = set_smem(var1a.fn[m], ba);
                if (st != FR_OK) return bail(st);
            }
            CUC(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&og, var1a.fn[1], var1a.threads, ba));
            if (og < 1) return bail(fail(ctx, FR_EUNSUPPORTED, "adjoint kernel does not fit on an SM"));
            ctx->Gg = std::min(ctx->U, og * sms);
        }
    }
    if (occ < 1) return bail(fail(ctx, FR_EUNSUPPORTED, "kernel does not fit on an SM"));
    ctx->G = std::min(ctx->U, occ * sms);
    if (!p2 && ctx->unrolled) ctx->Gg = std::min(ctx->Gg, ctx->G);  // gn2_part holds G partials
    ctx->nblk = reduce_blocks(ctx->I);

    const size_t ld = ctx->ld;
    if (p2) {
        CUC(cudaMalloc(&ctx->theta, sizeof(float) * ld));
        CUC(cudaMalloc(&ctx->tm1, sizeof(float) * ld));
        CUC(cudaMalloc(&ctx->tm2, sizeof(float) * ld));
        CUC(cudaMalloc(&ctx->w, sizeof(float) * ld));
        CUC(cudaMalloc(&ctx->gpart, sizeof(float) * (size_t)ctx->Gg * ld));
        if (ctx->unrolled) {
            const size_t nck = (size_t)ctx->U * ctx->nck * nc;
            CUC(cudaMalloc(&ctx->ck, sizeof(float) * nck));
            CUC(cudaMemset(ctx->ck, 0, sizeof(float) * nck));
            if (ctx->ce == 1) {  // state of the same size per iteration: the column sums too
                const size_t ncs = (size_t)ctx->U * ctx->cfg.sinkhorn_iters * nc;
                CUC(cudaMalloc(&ctx->csk, sizeof(float) * ncs));
                CUC(cudaMemset(ctx->csk, 0, sizeof(float) * ncs));
            }
        }
        CUC(cudaMalloc(&ctx->ad_blk, sizeof(double) * p2_adam_blocks(ctx->I)));
        CUC(cudaMalloc(&ctx->gn2_one, sizeof(double)));
    } else {
        const size_t cells = (size_t)ctx->U * nc * ld;
        if (ctx->unrolled) {
            CUC(cudaMalloc(&ctx->g0, sizeof(float) * (size_t)ctx->U * nc));
            CUC(cudaMemset(ctx->g0, 0, sizeof(float) * (size_t)ctx->U * nc));
            if (ctx->ce == 1) {  // the sweeps record every iteration; the adjoint only reverses
                const size_t n = (size_t)ctx->U * ctx->cfg.sinkhorn_iters * nc;
                CUC(cudaMalloc(&ctx->gall, sizeof(float) * n));
                CUC(cudaMalloc(&ctx->csall, sizeof(float) * n));
                CUC(cudaMemset(ctx->gall, 0, sizeof(float) * n));
                CUC(cudaMemset(ctx->csall, 0, sizeof(float) * n));
            }
        }
        CUC(cudaMalloc(&ctx->C, sizeof(float) * cells));
        CUC(cudaMalloc(&ctx->m1, sizeof(float) * cells));
        CUC(cudaMalloc(&ctx->m2, sizeof(float) * cells));
    }
    const size_t rbytes = (size_t)ctx->U * ld * (ctx->r_bf16 ? 2 : 4);
    CUC(cudaMalloc(&ctx->r, rbytes));
    CUC(cudaMemset(ctx->r, 0, rbytes));
    CUC(cudaMalloc(&ctx->gL, sizeof(float) * ctx->U * nc));
    CUC(cudaMalloc(&ctx->gP, sizeof(float) * ctx->U * nc));
    CUC(cudaMalloc(&ctx->e, sizeof(float) * nc));
    CUC(cudaMalloc(&ctx->invb, sizeof(float) * nc));
    CUC(cudaMalloc(&ctx->omega, sizeof(float) * ld));
    CUC(cudaMemset(ctx->omega, 0, sizeof(float) * ld));
    CUC(cudaMalloc(&ctx->part, sizeof(float) * (size_t)ctx->G * ld));
    CUC(cudaMalloc(&ctx->gn2_part, sizeof(double) * ctx->G));
    CUC(cudaMalloc(&ctx->imp, sizeof(double) * ld));
    CUC(cudaMalloc(&ctx->blk, sizeof(double) * 2 * ctx->nblk));
    CUC(cudaMalloc(&ctx->st, sizeof(DevState)));
    CUC(cudaMalloc(&ctx->flags, sizeof(int) * 4));
    CUC(cudaMallocHost(&ctx->st_host, sizeof(DevState)));
#undef CUC
    fr_status st = zero_state(ctx);
    if (st != FR_OK) return bail(st);
    st = ensure_hist(ctx, 64);
    if (st != FR_OK) return bail(st);
    *out = ctx;
    return FR_OK;
}

fr_status fr_destroy(fr_ctx* ctx) {
    if (!ctx) return FR_OK;
    cudaStreamSynchronize(ctx->s);
    free_all(ctx);
    delete ctx;
    return FR_OK;
}

fr_status fr_reset(fr_ctx* ctx) {
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    Join j(ctx);
    return zero_state(ctx);
}

fr_status fr_set_relevance(fr_ctx* ctx, const void* r, int32_t dtype, int64_t ld, int32_t on_device) {
    NvtxRange nvtx_range("fr_set_relevance");
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    if (!r) return fail(ctx, FR_EINVAL, "r is NULL");
    if (dtype != FR_F32 && dtype != FR_F64 && dtype != FR_BF16)
        return fail(ctx, FR_EINVAL, "unknown dtype %d", dtype);
    if (ld < ctx->I) return fail(ctx, FR_EINVAL, "ld %lld < n_items %d", (long long)ld, ctx->I);
    Join j(ctx);
    const size_t esz = dtype == FR_F64 ? 8 : dtype == FR_F32 ? 4 : 2;
    const void* src = r;
    int64_t lds = ld;
    if (!on_device) {
        fr_status st = ensure_tmp(ctx, esz * (size_t)ctx->U * ctx->I);
        if (st != FR_OK) return st;
        CU(cudaMemcpy2DAsync(ctx->tmp, esz * ctx->I, r, esz * ld, esz * ctx->I, ctx->U,
                             cudaMemcpyHostToDevice, ctx->s));
        src = ctx->tmp;
        lds = ctx->I;
    }
    CU(launch_relevance_import(src, dtype, lds, ctx->r, ctx->r_bf16, ctx->U, ctx->I, ctx->ld, ctx->s));
    CU(cudaMemsetAsync(ctx->flags, 0, sizeof(int) * 4, ctx->s));
    CU(launch_relevance_check(ctx->r, ctx->r_bf16, ctx->U, ctx->I, ctx->ld, ctx->flags, ctx->s));
    ctx->launches += 2;
    int hf[4];
    CU(cudaMemcpyAsync(hf, ctx->flags, sizeof hf, cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    if (hf[0]) return fail(ctx, FR_EINVAL, "relevance must be finite and >= 0");
    if (hf[1])
        return fail(ctx, FR_EINVAL, "%d items have no positive relevance (log Imp_i undefined)", hf[1]);
    ctx->have_r = true;
    ctx->fresh = false;
    return FR_OK;
}

fr_status fr_set_exposure(fr_ctx* ctx, const double* e, int32_t K) {
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    if (!e) return fail(ctx, FR_EINVAL, "e is NULL");
    if (K != ctx->K) return fail(ctx, FR_EINVAL, "K %d != n_slots %d", K, ctx->K);
    std::vector<float> ep(ctx->nc, 0.f), lb(ctx->nc, 1.f);  // lb: 1 / b_k
    float emax = 0.f;
    for (int k = 0; k < K; ++k) {
        if (!(e[k] > 0.0) || !std::isfinite(e[k]))
            return fail(ctx, FR_EINVAL, "exposure e[%d] must be positive and finite", k);
        ep[k] = (float)e[k];
        emax = std::max(emax, ep[k]);
    }
    if (ctx->nc > K) lb[K] = (float)(1.0 / (double)(ctx->I - K));  // dummy mass |I| - K
    Join j(ctx);
    CU(cudaMemcpyAsync(ctx->e, ep.data(), sizeof(float) * ctx->nc, cudaMemcpyHostToDevice, ctx->s));
    CU(cudaMemcpyAsync(ctx->invb, lb.data(), sizeof(float) * ctx->nc, cudaMemcpyHostToDevice, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    ctx->emax = emax;
    ctx->esum = 0.0;
    for (int k = 0; k < K; ++k) ctx->esum += e[k];
    ctx->have_e = true;
    ctx->fresh = false;
    return FR_OK;
}

fr_status fr_step(fr_ctx* ctx, int32_t n_steps, double* nsw_trace) {
    NvtxRange nvtx_range("fr_step");
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    if (n_steps < 0) return fail(ctx, FR_EINVAL, "n_steps < 0");
    Join j(ctx);
    fr_status st = ensure_fresh(ctx);
    if (st != FR_OK) return st;
    ctx->hist_n = 0;
    if ((st = ensure_hist(ctx, n_steps)) != FR_OK) return st;
    if ((st = set_run_state(ctx, -1.0)) != FR_OK) return st;
    if ((st = run_steps(ctx, n_steps)) != FR_OK) return st;
    if ((st = read_state(ctx)) != FR_OK) return st;
    ctx->hist_n = n_steps;
    if (nsw_trace && n_steps > 0) {
        CU(cudaMemcpyAsync(nsw_trace, ctx->F_hist, sizeof(double) * n_steps, cudaMemcpyDeviceToHost,
                           ctx->s));
        CU(cudaStreamSynchronize(ctx->s));
    }
    return FR_OK;
}

fr_status fr_solve(fr_ctx* ctx, double t, int32_t max_steps, int32_t* steps_done, double* nsw_out) {
    NvtxRange nvtx_range("fr_solve");
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    if (max_steps < 0 || !(t >= 0.0)) return fail(ctx, FR_EINVAL, "need max_steps >= 0 and t >= 0");
    Join j(ctx);
    fr_status st = ensure_fresh(ctx);
    if (st != FR_OK) return st;
    ctx->hist_n = 0;
    if ((st = ensure_hist(ctx, max_steps)) != FR_OK) return st;
    if ((st = set_run_state(ctx, t, max_steps)) != FR_OK) return st;
    if (max_steps > 0) {
        if ((st = ensure_solve_graph(ctx)) != FR_OK) return st;
        const int ctl[2] = {0, (max_steps + kChunk - 1) / kChunk};  // hard cap on body iterations
        CU(cudaMemcpyAsync(ctx->solve_ctl, ctl, sizeof ctl, cudaMemcpyHostToDevice, ctx->s));
        CU(cudaGraphLaunch(ctx->solve_exec, ctx->s));
        int done_ctl[2];
        CU(cudaMemcpyAsync(done_ctl, ctx->solve_ctl, sizeof done_ctl, cudaMemcpyDeviceToHost, ctx->s));
        CU(cudaStreamSynchronize(ctx->s));
        ctx->launches += (int64_t)done_ctl[0] * (kernels_per_step(ctx) * kChunk + 1);
    }
    if ((st = read_state(ctx)) != FR_OK) return st;
    ctx->hist_n = ctx->st_host->steps_done;
    if (steps_done) *steps_done = ctx->st_host->steps_done;
    if (nsw_out) *nsw_out = ctx->st_host->F;
    return set_run_state(ctx, -1.0);
}

fr_status fr_trace(fr_ctx* ctx, int32_t n, double* nsw, double* grad_norm, int32_t* n_steps) {
    NvtxRange nvtx_range("fr_trace");
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    if (n < 0) return fail(ctx, FR_EINVAL, "n < 0");
    const int m = std::min(n, ctx->hist_n);
    if (n_steps) *n_steps = ctx->hist_n;
    if (m == 0) return FR_OK;
    Join j(ctx);
    if (nsw) CU(cudaMemcpyAsync(nsw, ctx->F_hist, sizeof(double) * m, cudaMemcpyDeviceToHost, ctx->s));
    if (grad_norm)
        CU(cudaMemcpyAsync(grad_norm, ctx->gn_hist, sizeof(double) * m, cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    return FR_OK;
}

fr_status fr_impacts(fr_ctx* ctx, double* imp_out, double* utility_out, double* nsw_out) {
    NvtxRange nvtx_range("fr_impacts");
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    Join j(ctx);
    fr_status st = ensure_fresh(ctx);
    if (st != FR_OK) return st;
    if (imp_out)
        CU(cudaMemcpyAsync(imp_out, ctx->imp, sizeof(double) * ctx->I, cudaMemcpyDeviceToHost, ctx->s));
    if ((st = read_state(ctx)) != FR_OK) return st;
    if (utility_out) *utility_out = ctx->st_host->utility;
    if (nsw_out) *nsw_out = ctx->st_host->F;
    return FR_OK;
}

fr_status fr_policy(fr_ctx* ctx, int32_t u0, int32_t n_u, float* x_out, int32_t on_device) {
    NvtxRange nvtx_range("fr_policy");
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    if (u0 < 0 || n_u < 0 || (int64_t)u0 + n_u > ctx->U)
        return fail(ctx, FR_EINVAL, "consumer range [%d, %d) outside [0, %d)", u0, u0 + n_u, ctx->U);
    if (!x_out && n_u > 0) return fail(ctx, FR_EINVAL, "x_out is NULL");
    Join j(ctx);
    fr_status st = ensure_fresh(ctx);
    if (st != FR_OK) return st;
    const size_t bytes = sizeof(float) * (size_t)n_u * ctx->I * ctx->nc;
    float* dst = x_out;
    if (!on_device) {
        if ((st = ensure_tmp(ctx, bytes)) != FR_OK) return st;
        dst = ctx->tmp;
    }
    if (ctx->p2)
        CU(launch_p2_policy(p2_args(ctx, ctx->part), u0, n_u, dst, ctx->s));
    else
        CU(launch_policy(p1_args(ctx), u0, n_u, dst, ctx->s));
    ctx->launches += n_u > 0;
    if (!on_device && n_u > 0) CU(cudaMemcpyAsync(x_out, dst, bytes, cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    return FR_OK;
}

fr_status fr_grad(fr_ctx* ctx, const float* omega, float* dparam, float* dr, int32_t on_device) {
    NvtxRange nvtx_range("fr_grad");
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    if (!dparam) return fail(ctx, FR_EINVAL, "dparam is NULL");
    Join j(ctx);
    fr_status st = ensure_fresh(ctx);
    if (st != FR_OK) return st;
    const size_t nP = nparam(ctx), nr = (size_t)ctx->U * ctx->I;
    // staging: [omega (ld) | dparam (nP) | dr (nr)]
    const size_t need = sizeof(float) * (ctx->ld + (on_device ? 0 : nP + nr));
    if ((st = ensure_tmp(ctx, need)) != FR_OK) return st;
    const float* om = ctx->omega;
    if (omega) {
        CU(cudaMemsetAsync(ctx->tmp, 0, sizeof(float) * ctx->ld, ctx->s));
        CU(cudaMemcpyAsync(ctx->tmp, omega, sizeof(float) * ctx->I,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->s));
        om = ctx->tmp;
    }
    float* dP = on_device ? dparam : ctx->tmp + ctx->ld;
    float* dR = dr ? (on_device ? dr : ctx->tmp + ctx->ld + nP) : nullptr;
    if (ctx->p2) {
        P2Args a = p2_args(ctx, ctx->gpart);
        a.omega = om;
        a.dr = dR;
        CU(launch_p2_grad(ctx, a));
        CU(p2_launch_adam(adam_args(ctx, 0, dP), ctx->s));
        ctx->launches += 2;
    } else {
        P1Args a = p1_args(ctx);
        a.omega = om;
        a.dC = dP;
        a.dr = dR;
        if (ctx->unrolled)
            CU(p1_launch_adj(ctx->var1a, 0, a, ctx->Gg, ctx->s));
        else
            CU(p1_launch(ctx->var, MODE_GRAD, a, ctx->s));
        ctx->launches += 1;
    }
    if (!on_device) {
        CU(cudaMemcpyAsync(dparam, dP, sizeof(float) * nP, cudaMemcpyDeviceToHost, ctx->s));
        if (dr) CU(cudaMemcpyAsync(dr, dR, sizeof(float) * nr, cudaMemcpyDeviceToHost, ctx->s));
    }
    return read_state(ctx);  // synchronises; reports an expired wait of the gradient kernels
}

fr_status fr_set_state(fr_ctx* ctx, const float* param, const float* m1, const float* m2,
                       const float* g, int64_t t, int32_t on_device) {
    NvtxRange nvtx_range("fr_set_state");
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    if (t < 0) return fail(ctx, FR_EINVAL, "t < 0");
    Join j(ctx);
    const size_t nP = nparam(ctx);
    const float* srcs[3] = {param, m1, m2};
    float* dsts[3] = {ctx->p2 ? ctx->theta : ctx->C, ctx->p2 ? ctx->tm1 : ctx->m1,
                      ctx->p2 ? ctx->tm2 : ctx->m2};
    fr_status st = ensure_tmp(ctx, sizeof(float) * std::max(nP, (size_t)ctx->U * ctx->nc));
    if (st != FR_OK) return st;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    for (int q = 0; q < 3; ++q) {
        if (!srcs[q]) continue;
        if (ctx->p2) {  // [I] vectors, padding stays zero
            CU(cudaMemsetAsync(dsts[q], 0, sizeof(float) * ctx->ld, ctx->s));
            CU(cudaMemcpyAsync(dsts[q], srcs[q], sizeof(float) * ctx->I, kind, ctx->s));
        } else {
            const float* src = srcs[q];
            if (!on_device) {
                CU(cudaMemcpyAsync(ctx->tmp, src, sizeof(float) * nP, kind, ctx->s));
                src = ctx->tmp;
            }
            CU(launch_pack_ikn_to_kni(src, dsts[q], ctx->U, ctx->I, ctx->nc, ctx->ld, 1.f, ctx->s));
            ctx->launches += 1;
        }
    }
    if (ctx->p2 && param) {
        CU(launch_exp_theta(ctx->theta, ctx->w, ctx->I, ctx->ld, ctx->s));
        ctx->launches += 1;
    }
    if (g) {
        const float* src = g;
        if (!on_device) {
            CU(cudaMemcpyAsync(ctx->tmp, g, sizeof(float) * ctx->U * ctx->nc, kind, ctx->s));
            src = ctx->tmp;
        }
        CU(launch_scale(src, ctx->gL, (long long)ctx->U * ctx->nc,
                        (float)(1.0 / (ctx->cfg.epsilon * std::log(2.0))), ctx->s));
        ctx->launches += 1;
    }
    CU(cudaMemcpyAsync(ctx->st_host, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    ctx->st_host->t = t;
    CU(cudaMemcpyAsync(ctx->st, ctx->st_host, sizeof(DevState), cudaMemcpyHostToDevice, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    ctx->fresh = false;
    return FR_OK;
}

fr_status fr_get_state(fr_ctx* ctx, float* param, float* m1, float* m2, float* g, int64_t* t,
                       int32_t on_device) {
    NvtxRange nvtx_range("fr_get_state");
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    Join j(ctx);
    const size_t nP = nparam(ctx);
    float* dsts[3] = {param, m1, m2};
    const float* srcs[3] = {ctx->p2 ? ctx->theta : ctx->C, ctx->p2 ? ctx->tm1 : ctx->m1,
                            ctx->p2 ? ctx->tm2 : ctx->m2};
    fr_status st = ensure_tmp(ctx, sizeof(float) * std::max(nP, (size_t)ctx->U * ctx->nc));
    if (st != FR_OK) return st;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    for (int q = 0; q < 3; ++q) {
        if (!dsts[q]) continue;
        if (ctx->p2) {
            CU(cudaMemcpyAsync(dsts[q], srcs[q], sizeof(float) * ctx->I, kind, ctx->s));
        } else {
            float* dst = on_device ? dsts[q] : ctx->tmp;
            CU(launch_unpack_kni_to_ikn(srcs[q], dst, ctx->U, ctx->I, ctx->nc, ctx->ld, 1.f, ctx->s));
            ctx->launches += 1;
            if (!on_device) CU(cudaMemcpyAsync(dsts[q], dst, sizeof(float) * nP, kind, ctx->s));
        }
        CU(cudaStreamSynchronize(ctx->s));
    }
    if (g) {
        float* dst = on_device ? g : ctx->tmp;
        CU(launch_scale(ctx->gL, dst, (long long)ctx->U * ctx->nc,
                        (float)(ctx->cfg.epsilon * std::log(2.0)), ctx->s));
        ctx->launches += 1;
        if (!on_device)
            CU(cudaMemcpyAsync(g, dst, sizeof(float) * ctx->U * ctx->nc, kind, ctx->s));
    }
    CU(cudaMemcpyAsync(ctx->st_host, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    if (t) *t = ctx->st_host->t;
    return FR_OK;
}

// One evaluation of the Sec. 4.1 metrics; h receives mean envy, better %, worse %; env_host, when
// set, the per-item envy max_j (E_ij - E_ii) [I].
static fr_status metrics_run(fr_ctx* ctx, double h[3], double* env_host) {
    fr_status st = ensure_fresh(ctx);
    if (st != FR_OK) return st;
    // scratch in tmp: V [U][ld] floats | rmax [tiles][ld] floats | diag [ld] floats | ru [ld]
    // doubles | out [3] doubles | column-sum partials [colsum_chunks()][ld] doubles | per-item envy
    // [ld] doubles | the TF32 planes of R and V for the tensor cores (256-byte aligned pieces)
    const size_t ld = ctx->ld, nt = envy_tc_tiles(ctx->I);
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t oV = 0, oM = oV + al(4 * (size_t)ctx->U * ld), oD = oM + al(4 * nt * ld),
                 oR = oD + al(4 * ld), oO = oR + al(8 * ld), oP = oO + al(8 * 3),
                 oE = oP + al(8 * (size_t)colsum_chunks() * ld), oT = oE + al(8 * ld),
                 need = oT + al(envy_tc_plane_bytes(ctx->U, ctx->I));
    if ((st = ensure_tmp(ctx, need)) != FR_OK) return st;
    unsigned char* base = reinterpret_cast<unsigned char*>(ctx->tmp);
    float* V = reinterpret_cast<float*>(base + oV);
    double* out = reinterpret_cast<double*>(base + oO);
    double* env = env_host ? reinterpret_cast<double*>(base + oE) : nullptr;
    if (ctx->p2)
        CU(launch_v_p2(p2_args(ctx, ctx->part), V, ctx->s));
    else
        CU(launch_v_p1(p1_args(ctx), V, ctx->s));
    CU(cudaMemsetAsync(ctx->flags, 0, sizeof(int) * 4, ctx->s));
    CU(launch_envy(ctx->r, ctx->r_bf16, V, ctx->U, ctx->I, ctx->ld, ctx->imp, ctx->esum,
                   reinterpret_cast<float*>(base + oM), reinterpret_cast<float*>(base + oD),
                   reinterpret_cast<double*>(base + oR), reinterpret_cast<double*>(base + oP), out,
                   env, ctx->flags, polls_of(ctx->cfg.max_wait_polls), base + oT, ctx->s));
    ctx->launches += 7;
    int hf[4];
    CU(cudaMemcpyAsync(h, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->s));
    if (env) CU(cudaMemcpyAsync(env_host, env, sizeof(double) * ctx->I, cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaMemcpyAsync(hf, ctx->flags, sizeof hf, cudaMemcpyDeviceToHost, ctx->s));
    if ((st = read_state(ctx)) != FR_OK) return st;
    if (hf[0] & 4) return fail(ctx, FR_ETIMEOUT, "a bounded wait of the envy contraction expired");
    return FR_OK;
}

fr_status fr_metrics(fr_ctx* ctx, double* utility, double* mean_envy, double* better_pct,
                     double* worse_pct) {
    NvtxRange nvtx_range("fr_metrics");
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    Join j(ctx);
    double h[3];
    fr_status st = metrics_run(ctx, h, nullptr);
    if (st != FR_OK) return st;
    if (utility) *utility = ctx->st_host->utility;
    if (mean_envy) *mean_envy = h[0];
    if (better_pct) *better_pct = h[1];
    if (worse_pct) *worse_pct = h[2];
    return FR_OK;
}

fr_status fr_item_envy(fr_ctx* ctx, double* envy) {
    NvtxRange nvtx_range("fr_item_envy");
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    if (!envy) return fail(ctx, FR_EINVAL, "envy is NULL");
    Join j(ctx);
    double h[3];
    return metrics_run(ctx, h, envy);
}

fr_status fr_certificate(fr_ctx* ctx, double* gap, double* col_residual) {
    NvtxRange nvtx_range("fr_certificate");
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    Join j(ctx);
    fr_status st = ensure_fresh(ctx);
    if (st != FR_OK) return st;
    int sms = 0;
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    const int G = cert_grid(ctx->U, sms);
    // scratch: gap partials [G] doubles | residual partials [G] floats | out [2] doubles
    const size_t oR = 8 * (size_t)G, oO = (oR + 4 * (size_t)G + 15) / 16 * 16;
    if ((st = ensure_tmp(ctx, oO + 16)) != FR_OK) return st;
    unsigned char* base = reinterpret_cast<unsigned char*>(ctx->tmp);
    double* out = reinterpret_cast<double*>(base + oO);
    if (ctx->p2) {
        const P2Args a = p2_args(ctx, ctx->part);
        CU(launch_certificate(nullptr, &a, ctx->imp, ctx->nc, ctx->I, G,
                              reinterpret_cast<double*>(base), reinterpret_cast<float*>(base + oR), out,
                              ctx->s));
    } else {
        const P1Args a = p1_args(ctx);
        CU(launch_certificate(&a, nullptr, ctx->imp, ctx->nc, ctx->I, G,
                              reinterpret_cast<double*>(base), reinterpret_cast<float*>(base + oR), out,
                              ctx->s));
    }
    ctx->launches += 2;
    double h[2];
    CU(cudaMemcpyAsync(h, out, sizeof h, cudaMemcpyDeviceToHost, ctx->s));
    if ((st = read_state(ctx)) != FR_OK) return st;
    if (gap) *gap = h[0];
    if (col_residual) *col_residual = h[1];
    return FR_OK;
}

fr_status fr_time_kernels(fr_ctx* ctx, int32_t n_steps, double* ms) {
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    if (n_steps < 1 || !ms) return fail(ctx, FR_EINVAL, "need n_steps >= 1 and ms");
    Join j(ctx);
    fr_status st = ensure_fresh(ctx);
    if (st != FR_OK) return st;
    if ((st = set_run_state(ctx, -1.0)) != FR_OK) return st;
    cudaEvent_t ev[4];
    for (auto& e : ev) CU(cudaEventCreate(&e));
    double acc[3] = {0.0, 0.0, 0.0};
    for (int s = 0; s < n_steps; ++s) {
        CU(cudaEventRecord(ev[0], ctx->s));
        if (ctx->p2) {  // [gradient + theta update] [Sinkhorn] [reduction]
            CU(launch_p2_grad(ctx, p2_args(ctx, ctx->gpart)));
            CU(p2_launch_adam(adam_args(ctx, 1, nullptr), ctx->s));
            CU(cudaEventRecord(ev[1], ctx->s));
            CU(p2_launch_sweep(ctx->var2, p2_args(ctx, ctx->part), ctx->s));
            CU(cudaEventRecord(ev[2], ctx->s));
            CU(reduce_launch(red_args(ctx, 1), ctx->s));
            CU(cudaEventRecord(ev[3], ctx->s));
            ctx->launches += 4;
        } else if (ctx->unrolled) {  // [adjoint + optimiser] [Sinkhorn] [reduction]
            CU(p1_launch_adj(ctx->var1a, 1, p1_args(ctx), ctx->Gg, ctx->s));
            CU(cudaEventRecord(ev[1], ctx->s));
            CU(p1_launch(ctx->var, MODE_SWEEP, p1_args(ctx), ctx->s));
            CU(cudaEventRecord(ev[2], ctx->s));
            CU(reduce_launch(red_args(ctx, 1), ctx->s));
            CU(cudaEventRecord(ev[3], ctx->s));
            ctx->launches += 3;
        } else {  // [fused step] [reduction] [Sinkhorn only, same costs]
            CU(p1_launch(ctx->var, MODE_UPDATE_SWEEP, p1_args(ctx), ctx->s));
            CU(cudaEventRecord(ev[1], ctx->s));
            CU(reduce_launch(red_args(ctx, 1), ctx->s));
            CU(cudaEventRecord(ev[2], ctx->s));
            CU(p1_launch(ctx->var, MODE_SWEEP, p1_args(ctx), ctx->s));
            CU(cudaEventRecord(ev[3], ctx->s));
            CU(reduce_launch(red_args(ctx, 0), ctx->s));
            ctx->launches += 4;
        }
        CU(cudaStreamSynchronize(ctx->s));
        float a = 0.f, b = 0.f, c = 0.f;
        CU(cudaEventElapsedTime(&a, ev[0], ev[1]));
        CU(cudaEventElapsedTime(&b, ev[1], ev[2]));
        CU(cudaEventElapsedTime(&c, ev[2], ev[3]));
        if (ctx->p2 || ctx->unrolled) {
            acc[0] += b;  // Sinkhorn kernel
            acc[1] += c;  // reduction
            acc[2] += a;  // gradient + theta update
        } else {
            acc[0] += a;
            acc[1] += b;
            acc[2] += c;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    ms[0] = acc[0] / n_steps;
    ms[1] = acc[1] / n_steps;
    ms[2] = acc[2] / n_steps;
    return read_state(ctx);
}

fr_status fr_measure_peaks(double* out, int32_t n) {
    fr_ctx* ctx = nullptr;
    if (!out || n < 1 || n > 6) return fail(nullptr, FR_EINVAL, "need out and 1 <= n <= 6");
    double v[6] = {0, 0, 0, 0, 0, 0};
    const fr_status s0 = fr_measure_ex2_rate(&v[0]);
    if (s0 != FR_OK) return s0;
    int dev = 0, sms = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float* sink = nullptr;
    unsigned long long* clk = nullptr;
    CU(cudaMalloc(&sink, sizeof(float) * sms * 8));
    if (cudaMalloc(&clk, sizeof(unsigned long long) * 2) != cudaSuccess) {
        cudaFree(sink);
        return fail(nullptr, FR_ENOMEM, "cudaMalloc of the probe's clock record failed");
    }
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    std::vector<double> mhz;
    cudaError_t e = cudaSuccess;
    // kind, CTAs per SM, threads, iterations, units per thread and iteration (bytes or FMAs)
    const int kinds[4][4] = {{0, 4, 256, 4096}, {1, 4, 256, 2048}, {2, 8, 256, 16384},
                             {3, 8, 256, 8192}};
    const double per_it[4] = {8.0 * 8, 8.0 * 16, 8.0, 16.0};
    for (int q = 0; q < 4 && e == cudaSuccess; ++q) {
        const int kind = kinds[q][0], blocks = sms * kinds[q][1], threads = kinds[q][2];
        const int iters = kinds[q][3];
        e = launch_peak_bench(kind, sink, blocks, threads, 64, clk, nullptr);  // warm-up
        if (e != cudaSuccess) break;
        cudaEventRecord(a);
        e = launch_peak_bench(kind, sink, blocks, threads, iters, clk, nullptr);
        cudaEventRecord(b);
        if (e != cudaSuccess) break;
        if ((e = cudaEventSynchronize(b)) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        unsigned long long hc[2] = {0, 0};
        if ((e = cudaMemcpy(hc, clk, sizeof hc, cudaMemcpyDeviceToHost)) != cudaSuccess) break;
        if (hc[1] > 0) mhz.push_back((double)hc[0] / (double)hc[1] * 1e3);
        v[1 + q] = (double)blocks * threads * (double)iters * per_it[q] / (ms * 1e-3);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    cudaFree(clk);
    CU(e);
    if (!mhz.empty()) {
        std::sort(mhz.begin(), mhz.end());
        v[5] = mhz[mhz.size() / 2];
    }
    for (int j = 0; j < n; ++j) out[j] = v[j];
    return FR_OK;
}

fr_status fr_set_wait_limit(fr_ctx* ctx, int32_t max_wait_polls) {
    if (!ctx) return fail(nullptr, FR_EINVAL, "ctx is NULL");
    if (max_wait_polls < -1)
        return fail(ctx, FR_EINVAL, "max_wait_polls must be >= -1 (got %d)", max_wait_polls);
    if (max_wait_polls == ctx->cfg.max_wait_polls) return FR_OK;
    CU(cudaStreamSynchronize(ctx->s));  // the captured graphs hold the old limit: recapture
    if (ctx->chunk_exec) {
        cudaGraphExecDestroy(ctx->chunk_exec);
        ctx->chunk_exec = nullptr;
    }
    if (ctx->solve_exec) {
        cudaGraphExecDestroy(ctx->solve_exec);
        ctx->solve_exec = nullptr;
    }
    ctx->cfg.max_wait_polls = max_wait_polls;
    return FR_OK;
}

const char* fr_last_error(const fr_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

int64_t fr_launch_count(const fr_ctx* ctx) { return ctx ? ctx->launches : 0; }

fr_status fr_kernel_variant(const fr_ctx* ctx, int32_t* out) {
    if (!ctx || !out) return fail(nullptr, FR_EINVAL, "ctx or out is NULL");
    if (ctx->p2) {
        const P2Variant& v = ctx->var2;
        const int32_t o[6] = {v.ncb, v.rows, v.exact, v.threads, 0, ctx->G};
        for (int j = 0; j < 6; ++j) out[j] = o[j];
    } else {
        const P1Variant& v = ctx->var;
        const int32_t o[6] = {v.ncb, v.rows, v.exact, v.threads, v.tile_stride, ctx->G};
        for (int j = 0; j < 6; ++j) out[j] = o[j];
    }
    return FR_OK;
}

fr_status fr_sweep_stats(fr_ctx* ctx, int64_t* log_form_solves) {
    if (!ctx || !log_form_solves) return fail(nullptr, FR_EINVAL, "ctx or out is NULL");
    Join j(ctx);
    CU(cudaMemcpyAsync(ctx->st_host, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->s));
    CU(cudaStreamSynchronize(ctx->s));
    *log_form_solves = (int64_t)ctx->st_host->log_solves;
    return FR_OK;
}

fr_status fr_check_log2_near1(double* out) {
    fr_ctx* ctx = nullptr;
    if (!out) return fail(nullptr, FR_EINVAL, "output is NULL");
    int dev = 0, sms = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    unsigned* d = nullptr;
    CU(cudaMalloc(&d, sizeof(unsigned) * 3));
    unsigned h[3] = {0u, 0u, 0u};
    cudaError_t e = cudaMemset(d, 0, sizeof h);
    if (e == cudaSuccess) e = launch_log2_check(d, sms * 4, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    CU(e);
    float f[2];
    std::memcpy(f, h, sizeof f);
    out[0] = f[0];
    out[1] = f[1];
    out[2] = (double)h[2];
    return FR_OK;
}

fr_status fr_measure_ex2_rate(double* ex2_per_second) {
    fr_ctx* ctx = nullptr;
    if (!ex2_per_second) return fail(nullptr, FR_EINVAL, "output is NULL");
    int dev = 0, sms = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float* sink = nullptr;
    CU(cudaMalloc(&sink, sizeof(float) * sms * 8));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int blocks = sms * 8, threads = 256, iters = 4096;
    launch_ex2_bench(sink, blocks, threads, 64, nullptr);  // warm-up
    cudaEventRecord(a);
    launch_ex2_bench(sink, blocks, threads, iters, nullptr);
    cudaEventRecord(b);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    CU(e);
    *ex2_per_second = (double)blocks * threads * iters * 8.0 / (ms * 1e-3);
    return FR_OK;
}

}  // extern "C"
