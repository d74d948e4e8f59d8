// fr_batch.cu -- many independent markets (each its own instance of Problem (8), all under the
// per-item parametrisation or all with free costs) advanced together: the extern "C" fr_batch_*
// entry points of include/fairrank.h.
//
// Free-cost markets: a bucket is one kernel variant of the fused step kernel (column count, rows
// per thread, tile stride), its markets' consumers are cut into chunks with their own partial rows
// and squared-gradient partials, and per ascent step every bucket runs one persistent launch of the
// batched step kernel (gradient, Adam on the costs, Sinkhorn; concurrent branches) followed by one
// batched impact reduction. The autotuner chooses the chunk length per bucket. The rest of this
// header describes the per-item markets.
//
// Markets are grouped into buckets that share one kernel shape: the column count the kernel is
// compiled for (exactly 6, 11 or 21 columns, or a padded 8 / 16 / 32 bucket) and the CTA size
// (warps needed at 8 rows per thread). Every bucket's consumers are cut into chunks (a run of
// consumers of one market with its own partial row), and one persistent launch per bucket walks the
// chunk list. Per ascent step the launches are: the gradient of every bucket (concurrent graph
// branches), one batched theta update over all markets, the Sinkhorn sweep of every bucket
// (concurrent branches) and one batched impact reduction; chunks of steps are replayed as one CUDA
// graph. An autotuner times the rows-per-thread and chunk-length candidates of each bucket on the
// bucket's own data before the first solve and keeps the fastest.
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
constexpr int kBatchChunk = 8;     // ascent steps per captured graph
constexpr int kMaxSide = 8;        // side streams for concurrent bucket launches
constexpr int kCpcCand[] = {4, 16};  // consumers per chunk, autotuner candidates
constexpr int kCpcMin = 4;
thread_local std::string g_batch_create_error;
}  // namespace

struct BMarket {
    int U = 0, I = 0, K = 0, nc = 0, ld = 0, rows = 0, bucket = -1;
    float emax = 0.f;
    bool have_r = false, have_e = false;
    void* r = nullptr;
    float *C = nullptr, *m1 = nullptr, *m2 = nullptr;  // free costs: C and Adam moments [U][nc][ld]
    float *theta = nullptr, *tm1 = nullptr, *tm2 = nullptr, *w = nullptr, *gL = nullptr,
          *gP = nullptr, *e = nullptr, *invb = nullptr, *omega = nullptr, *part = nullptr,
          *gpart = nullptr;
    double *imp = nullptr, *blk = nullptr, *ad_blk = nullptr, *gn2 = nullptr, *F_hist = nullptr,
           *gn_hist = nullptr;
    DevState* st = nullptr;
};

struct BBucket {
    int ncb = 0, exact = 0, warps8 = 0, I_max = 0, ld_max = 0;
    std::vector<int> markets;
    P2Variant var{};
    // free costs: the batched kernel variant (rows per thread and tile stride fixed by the variant
    // table), its shared memory and occupancy-bound grids for MODE_SWEEP / MODE_UPDATE_SWEEP
    P1Variant var1{};
    int tile_stride = 0, threads1 = 0;
    size_t smem1[2] = {0, 0};
    int G1[2] = {0, 0};
    int R = 8, cpc = kCpcMin, n_chunks = 0, G_sweep = 0, G_grad = 0, occ_sweep = 0, occ_grad = 0;
    P2Chunk* d_chunks = nullptr;
    size_t smem_sweep = 0, smem_grad = 0;
};

struct fr_batch {
    fr_config cfg{};  // shared fields (sizes of market 0)
    bool p1 = false;  // free-cost markets (FR_PARAM_FULL_C), else per-item variables
    P1Args* d_args_p1 = nullptr;
    int M = 0, device = 0, sms = 0, max_optin = 0;
    int esz = 4;
    std::vector<BMarket> mk;
    std::vector<BBucket> bk;
    P2Args* d_args_sweep = nullptr;
    P2Args* d_args_grad = nullptr;
    ReduceArgs* d_red = nullptr;   // after an update (gradient norm, history, t)
    ReduceArgs* d_red0 = nullptr;  // after a plain solve
    P2AdamArgs* d_adam = nullptr;
    int2* d_red_map = nullptr;
    int2* d_adam_map = nullptr;
    int n_red_blocks = 0, n_adam_blocks = 0;
    int hist_cap = 0;
    void* arena = nullptr;       // all per-market buffers except the history
    void* hist_arena = nullptr;  // F and gradient-norm histories
    DevState* st_host = nullptr; // pinned [M]
    int* flags = nullptr;
    float* tmp = nullptr;
    size_t tmp_bytes = 0;
    cudaStream_t user = nullptr, s = nullptr;
    cudaStream_t side[kMaxSide] = {};
    int nside = 0;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr;
    cudaEvent_t ev_join[kMaxSide] = {};
    cudaGraphExec_t chunk_exec = nullptr;
    bool tuned = false, fresh = false;
    int64_t launches = 0;
    std::string err;
};

namespace {

fr_status bfail(fr_batch* b, fr_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b)
        b->err = buf;
    else
        g_batch_create_error = buf;
    return st;
}

#define BCU(call)                                                                             \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            cudaGetLastError(); /* no stale error in a later call's checks */                 \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? FR_ENOMEM : FR_ECUDA, "%s: %s", \
                         #call, cudaGetErrorString(e_));                                      \
        }                                                                                     \
    } while (0)

struct BJoin {
    fr_batch* b;
    explicit BJoin(fr_batch* bb) : b(bb) {
        cudaEventRecord(b->ev_in, b->user);
        cudaStreamWaitEvent(b->s, b->ev_in, 0);
    }
    ~BJoin() {
        cudaEventRecord(b->ev_out, b->s);
        cudaStreamWaitEvent(b->user, b->ev_out, 0);
    }
};

int warps_at(int I, int R) { return ((I + R - 1) / R + 31) / 32; }

int ncb_of(int nc) {
    if (nc == 21 || nc == 11 || nc == 6) return nc;
    return nc <= 8 ? 8 : (nc <= 16 ? 16 : 32);
}

bool variant_for(int ncb, int R, int threads, P2Variant* v) {
    if (ncb == 21) return p2_variant_k21(R, threads, v);
    if (ncb == 11) return p2_variant_k11(R, threads, v);
    if (ncb == 6) return p2_variant_k6(R, threads, v);
    if (R != 8) return false;
    return p2_variant_generic(ncb, threads, v);
}

P2Args market_args(const fr_batch* b, const BMarket& m, float* part) {
    P2Args a{};
    a.U = m.U; a.I = m.I; a.K = m.K; a.nc = m.nc; a.ld = m.ld; a.L = b->cfg.sinkhorn_iters;
    a.G = m.rows;
    a.r = m.r; a.r_bf16 = b->esz == 2; a.w = m.w; a.e = m.e; a.invb = m.invb; a.emax = m.emax;
    a.gL = m.gL; a.gP = m.gP; a.part = part; a.omega = m.omega; a.dr = nullptr; a.st = m.st;
    a.inv_eps_ln2 = (float)(1.0 / (b->cfg.epsilon * std::log(2.0)));
    a.inv_eps = (float)(1.0 / b->cfg.epsilon);
    a.warm = b->cfg.warm_start ? 1 : 0;
    a.max_polls = polls_of(b->cfg.max_wait_polls);
    return a;
}

// Free costs: the arguments of market m's step kernels (one partial row and one squared-gradient
// partial per chunk).
P1Args market_args_p1(const fr_batch* b, const BMarket& m) {
    P1Args a{};
    a.U = m.U; a.I = m.I; a.K = m.K; a.nc = m.nc; a.ld = m.ld; a.L = b->cfg.sinkhorn_iters;
    a.G = m.rows;
    a.C = m.C; a.m1 = m.m1; a.m2 = m.m2; a.gL = m.gL; a.gP = m.gP;
    a.r = static_cast<const float*>(m.r); a.e = m.e; a.invb = m.invb; a.omega = m.omega;
    a.part = m.part; a.gn2_part = m.gn2; a.st = m.st;
    a.inv_eps_ln2 = (float)(1.0 / (b->cfg.epsilon * std::log(2.0)));
    a.inv_eps = (float)(1.0 / b->cfg.epsilon);
    a.lr = (float)b->cfg.lr; a.beta1 = (float)b->cfg.beta1; a.beta2 = (float)b->cfg.beta2;
    a.adam_eps = (float)b->cfg.adam_eps;
    a.optimizer = b->cfg.optimizer == FR_SGD ? 1 : 0;
    a.warm = b->cfg.warm_start ? 1 : 0;
    a.max_polls = polls_of(b->cfg.max_wait_polls);
    return a;
}

fr_status upload_tables_p1(fr_batch* b) {
    std::vector<P1Args> a1(b->M);
    std::vector<ReduceArgs> ra(b->M);
    for (int i = 0; i < b->M; ++i) {
        BMarket& m = b->mk[i];
        const BBucket& k = b->bk[m.bucket];
        m.rows = (m.U + k.cpc - 1) / k.cpc;
        a1[i] = market_args_p1(b, m);
        ReduceArgs& r = ra[i];
        r = ReduceArgs{};
        r.I = m.I; r.ld = m.ld; r.G = m.rows; r.U = m.U; r.Ggn = m.rows;
        r.part = m.part; r.gn2_part = m.gn2; r.imp = m.imp; r.omega = m.omega; r.blk = m.blk;
        r.st = m.st; r.F_hist = m.F_hist; r.gn_hist = m.gn_hist; r.hist_cap = b->hist_cap;
        r.after_update = 1; r.nblk = reduce_blocks(m.I);
    }
    BCU(cudaMemcpyAsync(b->d_args_p1, a1.data(), sizeof(P1Args) * b->M, cudaMemcpyHostToDevice, b->s));
    BCU(cudaMemcpyAsync(b->d_red, ra.data(), sizeof(ReduceArgs) * b->M, cudaMemcpyHostToDevice, b->s));
    for (auto& r : ra) r.after_update = 0;
    BCU(cudaMemcpyAsync(b->d_red0, ra.data(), sizeof(ReduceArgs) * b->M, cudaMemcpyHostToDevice, b->s));
    BCU(cudaStreamSynchronize(b->s));
    return FR_OK;
}

// Device argument tables (market arguments, reduction and update arguments) from the host state;
// the partial-row counts follow each bucket's chosen chunk length.
fr_status upload_tables(fr_batch* b) {
    if (b->p1) return upload_tables_p1(b);
    std::vector<P2Args> as(b->M), ag(b->M);
    std::vector<ReduceArgs> ra(b->M);
    std::vector<P2AdamArgs> aa(b->M);
    for (int i = 0; i < b->M; ++i) {
        BMarket& m = b->mk[i];
        const BBucket& k = b->bk[m.bucket];
        m.rows = (m.U + k.cpc - 1) / k.cpc;
        as[i] = market_args(b, m, m.part);
        ag[i] = market_args(b, m, m.gpart);
        ReduceArgs& r = ra[i];
        r = ReduceArgs{};
        r.I = m.I; r.ld = m.ld; r.G = m.rows; r.U = m.U; r.Ggn = 1;
        r.part = m.part; r.gn2_part = m.gn2; r.imp = m.imp; r.omega = m.omega; r.blk = m.blk;
        r.st = m.st; r.F_hist = m.F_hist; r.gn_hist = m.gn_hist; r.hist_cap = b->hist_cap;
        r.after_update = 1; r.nblk = reduce_blocks(m.I);
        P2AdamArgs& d = aa[i];
        d = P2AdamArgs{};
        d.I = m.I; d.ld = m.ld; d.G = m.rows; d.part = m.gpart; d.theta = m.theta; d.m1 = m.tm1;
        d.m2 = m.tm2; d.w = m.w; d.dtheta_out = nullptr; d.gn2_out = m.gn2; d.blk = m.ad_blk;
        d.st = m.st; d.lr = (float)b->cfg.lr; d.beta1 = (float)b->cfg.beta1;
        d.beta2 = (float)b->cfg.beta2; d.adam_eps = (float)b->cfg.adam_eps;
        d.optimizer = b->cfg.optimizer == FR_SGD ? 1 : 0; d.apply = 1;
        d.nblk = p2_adam_blocks(m.I);
    }
    BCU(cudaMemcpyAsync(b->d_args_sweep, as.data(), sizeof(P2Args) * b->M, cudaMemcpyHostToDevice, b->s));
    BCU(cudaMemcpyAsync(b->d_args_grad, ag.data(), sizeof(P2Args) * b->M, cudaMemcpyHostToDevice, b->s));
    BCU(cudaMemcpyAsync(b->d_red, ra.data(), sizeof(ReduceArgs) * b->M, cudaMemcpyHostToDevice, b->s));
    for (auto& r : ra) r.after_update = 0;
    BCU(cudaMemcpyAsync(b->d_red0, ra.data(), sizeof(ReduceArgs) * b->M, cudaMemcpyHostToDevice, b->s));
    BCU(cudaMemcpyAsync(b->d_adam, aa.data(), sizeof(P2AdamArgs) * b->M, cudaMemcpyHostToDevice, b->s));
    BCU(cudaStreamSynchronize(b->s));
    return FR_OK;
}

// Chunk list of a bucket for chunk length cpc: runs of cpc consumers, longest work first (LPT
// order over the persistent CTAs' round-robin), each with its market's next partial row.
std::vector<P2Chunk> make_chunks(const fr_batch* b, const BBucket& k, int cpc) {
    std::vector<P2Chunk> ch;
    for (int mi : k.markets) {
        const BMarket& m = b->mk[mi];
        int row = 0;
        for (int u = 0; u < m.U; u += cpc, ++row) ch.push_back({mi, u, std::min(u + cpc, m.U), row});
    }
    std::stable_sort(ch.begin(), ch.end(), [&](const P2Chunk& x, const P2Chunk& y) {
        const double cx = (double)(x.u1 - x.u0) * b->mk[x.market].I * b->mk[x.market].nc;
        const double cy = (double)(y.u1 - y.u0) * b->mk[y.market].I * b->mk[y.market].nc;
        return cx > cy;
    });
    return ch;
}

// Configures bucket k for (R, cpc): variant, shared memory, occupancy-bound grids, chunk list.
fr_status configure_bucket(fr_batch* b, BBucket& k, int R, int cpc) {
    const int threads = warps_at(k.I_max, R) * 32;
    if (threads > 512 || !variant_for(k.ncb, R, threads, &k.var))
        return bfail(b, FR_EUNSUPPORTED, "no kernel for %d columns, %d rows per thread, %d items",
                     k.ncb, R, k.I_max);
    k.R = R;
    k.cpc = cpc;
    k.smem_sweep = p2_sweep_smem_batch(k.var, k.ld_max, b->esz);
    k.smem_grad = p2_grad_smem_batch(k.var, k.ld_max, b->esz);
    if (k.smem_sweep > (size_t)b->max_optin || k.smem_grad > (size_t)b->max_optin)
        return bfail(b, FR_EUNSUPPORTED, "shared memory for %d items exceeds the device limit",
                     k.I_max);
    BCU(raise_smem_limit(k.var.sweep_b, k.smem_sweep));
    BCU(raise_smem_limit(k.var.grad_b, k.smem_grad));
    int o1 = 0, o2 = 0;
    BCU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k.var.sweep_b, threads, k.smem_sweep));
    BCU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k.var.grad_b, threads, k.smem_grad));
    if (o1 < 1 || o2 < 1) return bfail(b, FR_EUNSUPPORTED, "bucket kernel does not fit on an SM");
    const std::vector<P2Chunk> ch = make_chunks(b, k, cpc);
    k.n_chunks = (int)ch.size();
    k.occ_sweep = o1;
    k.occ_grad = o2;
    // every bucket's grid fills the GPU: concurrent launches of different shapes rarely share an
    // SM (each needs its own shared-memory carveout), so grids sized as shares of the SMs were
    // measured 3x slower than full grids whose tails overlap the next bucket's launch
    k.G_sweep = std::min(k.n_chunks, o1 * b->sms);
    k.G_grad = std::min(k.n_chunks, o2 * b->sms);
    cudaFree(k.d_chunks);
    k.d_chunks = nullptr;
    BCU(cudaMalloc(&k.d_chunks, sizeof(P2Chunk) * std::max<size_t>(ch.size(), 1)));
    BCU(cudaMemcpyAsync(k.d_chunks, ch.data(), sizeof(P2Chunk) * ch.size(), cudaMemcpyHostToDevice, b->s));
    BCU(cudaStreamSynchronize(b->s));
    return FR_OK;
}

// Free costs: configures bucket k for chunks of cpc consumers (the rows per thread and the tile
// stride come with the bucket's kernel variant).
fr_status configure_bucket_p1(fr_batch* b, BBucket& k, int cpc) {
    k.cpc = cpc;
    k.R = k.var1.rows;
    for (int m = 0; m < 2; ++m) {
        const int mode = m ? MODE_UPDATE_SWEEP : MODE_SWEEP;
        k.smem1[m] = p1_smem_bytes_batch(k.var1, mode, k.ld_max);
        if (k.smem1[m] > (size_t)b->max_optin)
            return bfail(b, FR_EUNSUPPORTED, "shared memory for %d items and %d columns exceeds the "
                         "device limit", k.I_max, k.ncb);
        BCU(raise_smem_limit(k.var1.fb[m], k.smem1[m]));
    }
    const std::vector<P2Chunk> ch = make_chunks(b, k, cpc);
    k.n_chunks = (int)ch.size();
    for (int m = 0; m < 2; ++m) {
        int o = 0;
        BCU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k.var1.fb[m], k.var1.threads, k.smem1[m]));
        if (o < 1) return bfail(b, FR_EUNSUPPORTED, "bucket kernel does not fit on an SM");
        k.G1[m] = std::min(k.n_chunks, o * b->sms);
    }
    cudaFree(k.d_chunks);
    k.d_chunks = nullptr;
    BCU(cudaMalloc(&k.d_chunks, sizeof(P2Chunk) * std::max<size_t>(ch.size(), 1)));
    BCU(cudaMemcpyAsync(k.d_chunks, ch.data(), sizeof(P2Chunk) * ch.size(), cudaMemcpyHostToDevice, b->s));
    BCU(cudaStreamSynchronize(b->s));
    return FR_OK;
}

P1Batch batch_of_p1(const fr_batch* b, const BBucket& k) {
    P1Batch bt{};
    bt.mk = b->d_args_p1;
    bt.ch = k.d_chunks;
    bt.n_chunks = k.n_chunks;
    bt.ld_max = k.ld_max;
    return bt;
}

// Free costs: one step kernel per bucket (MODE_SWEEP or MODE_UPDATE_SWEEP), buckets on the side
// streams.
fr_status launch_phase_p1(fr_batch* b, int mode) {
    BCU(cudaEventRecord(b->ev_fork, b->s));
    for (int j = 0; j < b->nside; ++j) BCU(cudaStreamWaitEvent(b->side[j], b->ev_fork, 0));
    for (size_t i = 0; i < b->bk.size(); ++i) {
        const BBucket& k = b->bk[i];
        BCU(p1_launch_batch(k.var1, mode, batch_of_p1(b, k), k.G1[mode == MODE_UPDATE_SWEEP],
                            b->side[i % b->nside]));
        b->launches += 1;
    }
    for (int j = 0; j < b->nside; ++j) {
        BCU(cudaEventRecord(b->ev_join[j], b->side[j]));
        BCU(cudaStreamWaitEvent(b->s, b->ev_join[j], 0));
    }
    return FR_OK;
}

P2Batch batch_of(const fr_batch* b, const BBucket& k, bool grad) {
    P2Batch bt{};
    bt.mk = grad ? b->d_args_grad : b->d_args_sweep;
    bt.ch = k.d_chunks;
    bt.n_chunks = k.n_chunks;
    bt.ld_max = k.ld_max;
    bt.esz = b->esz;
    return bt;
}

// One phase (gradient or sweep) of every bucket, buckets spread over the side streams.
fr_status launch_phase(fr_batch* b, bool grad) {
    BCU(cudaEventRecord(b->ev_fork, b->s));
    for (int j = 0; j < b->nside; ++j) BCU(cudaStreamWaitEvent(b->side[j], b->ev_fork, 0));
    for (size_t i = 0; i < b->bk.size(); ++i) {
        const BBucket& k = b->bk[i];
        cudaStream_t st = b->side[i % b->nside];
        if (grad)
            BCU(p2_launch_grad_batch(k.var, batch_of(b, k, true), k.G_grad, st));
        else
            BCU(p2_launch_sweep_batch(k.var, batch_of(b, k, false), k.G_sweep, st));
        b->launches += 1;
    }
    for (int j = 0; j < b->nside; ++j) {
        BCU(cudaEventRecord(b->ev_join[j], b->side[j]));
        BCU(cudaStreamWaitEvent(b->s, b->ev_join[j], 0));
    }
    return FR_OK;
}

fr_status launch_solve(fr_batch* b) {
    fr_status st = b->p1 ? launch_phase_p1(b, MODE_SWEEP) : launch_phase(b, false);
    if (st != FR_OK) return st;
    BCU(reduce_launch_batch(b->d_red0, b->d_red_map, b->n_red_blocks, b->s));
    b->launches += 1;
    return FR_OK;
}

fr_status launch_step(fr_batch* b) {
    if (b->p1) {  // fused gradient + Adam + Sinkhorn per bucket, then the impact reduction
        fr_status st = launch_phase_p1(b, MODE_UPDATE_SWEEP);
        if (st != FR_OK) return st;
        BCU(reduce_launch_batch(b->d_red, b->d_red_map, b->n_red_blocks, b->s));
        b->launches += 1;
        return FR_OK;
    }
    fr_status st = launch_phase(b, true);
    if (st != FR_OK) return st;
    BCU(p2_launch_adam_batch(b->d_adam, b->d_adam_map, b->n_adam_blocks, b->s));
    if ((st = launch_phase(b, false)) != FR_OK) return st;
    BCU(reduce_launch_batch(b->d_red, b->d_red_map, b->n_red_blocks, b->s));
    b->launches += 2;
    return FR_OK;
}

int kernels_per_step(const fr_batch* b) {
    return b->p1 ? (int)b->bk.size() + 1 : 2 * (int)b->bk.size() + 2;
}

fr_status ensure_graph(fr_batch* b) {
    if (b->chunk_exec) return FR_OK;
    cudaGraph_t g = nullptr;
    const int64_t before = b->launches;
    BCU(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
    for (int j = 0; j < kBatchChunk; ++j) {
        fr_status st = launch_step(b);
        if (st != FR_OK) {
            cudaStreamEndCapture(b->s, &g);
            if (g) cudaGraphDestroy(g);
            b->launches = before;
            return st;
        }
    }
    b->launches = before;  // captured, not launched
    BCU(cudaStreamEndCapture(b->s, &g));
    cudaError_t e = cudaGraphInstantiate(&b->chunk_exec, g, 0);
    cudaGraphDestroy(g);
    BCU(e);
    return FR_OK;
}

void drop_graph(fr_batch* b) {
    if (b->chunk_exec) cudaGraphExecDestroy(b->chunk_exec);
    b->chunk_exec = nullptr;
}

fr_status read_states(fr_batch* b) {
    BCU(cudaStreamSynchronize(b->s));
    for (int i = 0; i < b->M; ++i)
        BCU(cudaMemcpyAsync(b->st_host + i, b->mk[i].st, sizeof(DevState), cudaMemcpyDeviceToHost, b->s));
    BCU(cudaStreamSynchronize(b->s));
    for (int i = 0; i < b->M; ++i) {
        const int e = b->st_host[i].err;
        if (e & 4) return bfail(b, FR_ETIMEOUT, "market %d: a bounded wait for a staged bulk copy expired", i);
        if (e) return bfail(b, FR_ENUMERIC, "market %d: non-finite or non-positive impact (flags %d)", i, e);
    }
    return FR_OK;
}

fr_status set_run_states(fr_batch* b) {
    fr_status st = read_states(b);
    if (st != FR_OK) return st;
    for (int i = 0; i < b->M; ++i) {
        DevState& h = b->st_host[i];
        h.hist_idx = 0;
        h.stop = 0;
        h.steps_done = 0;
        h.thresh = -1.0;
        BCU(cudaMemcpyAsync(b->mk[i].st, &h, sizeof(DevState), cudaMemcpyHostToDevice, b->s));
    }
    BCU(cudaStreamSynchronize(b->s));
    return FR_OK;
}

fr_status ensure_hist(fr_batch* b, int n) {
    if (n <= b->hist_cap) return FR_OK;
    int cap = b->hist_cap > 0 ? b->hist_cap : 64;
    while (cap < n) cap *= 2;
    BCU(cudaStreamSynchronize(b->s));
    cudaFree(b->hist_arena);
    b->hist_arena = nullptr;
    BCU(cudaMalloc(&b->hist_arena, sizeof(double) * 2 * (size_t)cap * b->M));
    double* h = static_cast<double*>(b->hist_arena);
    for (int i = 0; i < b->M; ++i) {
        b->mk[i].F_hist = h + (size_t)2 * cap * i;
        b->mk[i].gn_hist = h + (size_t)2 * cap * i + cap;
    }
    b->hist_cap = cap;
    drop_graph(b);
    return upload_tables(b);
}

fr_status zero_state(fr_batch* b) {
    for (auto& m : b->mk) {
        if (b->p1) {  // C = 0 (the uniform policy) and zero moments
            const size_t cells = sizeof(float) * (size_t)m.U * m.nc * m.ld;
            BCU(cudaMemsetAsync(m.C, 0, cells, b->s));
            BCU(cudaMemsetAsync(m.m1, 0, cells, b->s));
            BCU(cudaMemsetAsync(m.m2, 0, cells, b->s));
        } else {
            BCU(cudaMemsetAsync(m.theta, 0, sizeof(float) * m.ld, b->s));
            BCU(cudaMemsetAsync(m.tm1, 0, sizeof(float) * m.ld, b->s));
            BCU(cudaMemsetAsync(m.tm2, 0, sizeof(float) * m.ld, b->s));
            BCU(launch_exp_theta(m.theta, m.w, m.I, m.ld, b->s));
        }
        BCU(cudaMemsetAsync(m.gL, 0, sizeof(float) * (size_t)m.U * m.nc, b->s));
        BCU(cudaMemsetAsync(m.gP, 0, sizeof(float) * (size_t)m.U * m.nc, b->s));
        DevState z{};
        z.thresh = -1.0;
        BCU(cudaMemcpyAsync(m.st, &z, sizeof(DevState), cudaMemcpyHostToDevice, b->s));
        BCU(cudaStreamSynchronize(b->s));
    }
    b->launches += b->M;
    b->fresh = false;
    return FR_OK;
}

// Times one sweep launch of bucket k (mean of `reps` after one warm-up) in milliseconds.
fr_status time_bucket(fr_batch* b, const BBucket& k, int reps, float* ms) {
    cudaEvent_t e0, e1;
    BCU(cudaEventCreate(&e0));
    BCU(cudaEventCreate(&e1));
    auto sweep = [&]() {
        return b->p1 ? p1_launch_batch(k.var1, MODE_SWEEP, batch_of_p1(b, k), k.G1[0], b->s)
                     : p2_launch_sweep_batch(k.var, batch_of(b, k, false), k.G_sweep, b->s);
    };
    BCU(sweep());
    BCU(cudaEventRecord(e0, b->s));
    for (int r = 0; r < reps; ++r) BCU(sweep());
    BCU(cudaEventRecord(e1, b->s));
    BCU(cudaEventSynchronize(e1));
    float t = 0.f;
    BCU(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->launches += reps + 1;
    *ms = t / reps;
    return FR_OK;
}

// For every bucket: time each (rows per thread, chunk length) candidate on the bucket's own markets
// and keep the fastest. The warm-start potentials are saved and restored around the trial sweeps.
fr_status autotune(fr_batch* b) {
    size_t gbytes = 0;
    for (auto& m : b->mk) gbytes += sizeof(float) * (size_t)m.U * m.nc;
    std::vector<float> saveL(gbytes / sizeof(float)), saveP(gbytes / sizeof(float));
    size_t off = 0;
    for (auto& m : b->mk) {
        const size_t n = (size_t)m.U * m.nc;
        BCU(cudaMemcpyAsync(saveL.data() + off, m.gL, sizeof(float) * n, cudaMemcpyDeviceToHost, b->s));
        BCU(cudaMemcpyAsync(saveP.data() + off, m.gP, sizeof(float) * n, cudaMemcpyDeviceToHost, b->s));
        off += n;
    }
    BCU(cudaStreamSynchronize(b->s));
    for (auto& k : b->bk) {
        if (b->p1) {  // free costs: the chunk length (rows per thread come with the variant)
            int bestC = kCpcMin;
            float best = 1e30f;
            for (int cpc : kCpcCand) {
                fr_status st = configure_bucket_p1(b, k, cpc);
                if (st != FR_OK) return st;
                if ((st = upload_tables(b)) != FR_OK) return st;
                float ms = 0.f;
                if ((st = time_bucket(b, k, 2, &ms)) != FR_OK) return st;
                if (ms < best) {
                    best = ms;
                    bestC = cpc;
                }
            }
            fr_status st = configure_bucket_p1(b, k, bestC);
            if (st != FR_OK) return st;
            continue;
        }
        int bestR = 8, bestC = kCpcMin;
        float best = 1e30f;
        const int Rs[] = {8, 16, 24};
        for (int R : Rs) {
            if (R != 8 && !k.exact) continue;
            if (warps_at(k.I_max, R) * 32 > 512) continue;
            if (R > 8 && warps_at(k.I_max, R) == warps_at(k.I_max, R - 8)) continue;  // same CTA
            for (int cpc : kCpcCand) {
                fr_status st = configure_bucket(b, k, R, cpc);
                if (st != FR_OK) return st;
                if ((st = upload_tables(b)) != FR_OK) return st;
                float ms = 0.f;
                if ((st = time_bucket(b, k, 2, &ms)) != FR_OK) return st;
                if (ms < best) {
                    best = ms;
                    bestR = R;
                    bestC = cpc;
                }
            }
        }
        fr_status st = configure_bucket(b, k, bestR, bestC);
        if (st != FR_OK) return st;
    }
    fr_status st = upload_tables(b);
    if (st != FR_OK) return st;
    off = 0;
    for (auto& m : b->mk) {
        const size_t n = (size_t)m.U * m.nc;
        BCU(cudaMemcpyAsync(m.gL, saveL.data() + off, sizeof(float) * n, cudaMemcpyHostToDevice, b->s));
        BCU(cudaMemcpyAsync(m.gP, saveP.data() + off, sizeof(float) * n, cudaMemcpyHostToDevice, b->s));
        off += n;
    }
    BCU(cudaStreamSynchronize(b->s));
    drop_graph(b);
    b->tuned = true;
    b->fresh = false;
    return FR_OK;
}

fr_status ensure_ready(fr_batch* b) {
    for (int i = 0; i < b->M; ++i)
        if (!b->mk[i].have_r || !b->mk[i].have_e)
            return bfail(b, FR_ESTATE, "market %d: set relevance and exposure first", i);
    fr_status st = FR_OK;
    if (!b->tuned && (st = autotune(b)) != FR_OK) return st;
    if (!b->fresh) {
        if ((st = set_run_states(b)) != FR_OK) return st;
        if ((st = launch_solve(b)) != FR_OK) return st;
        b->fresh = true;
    }
    return FR_OK;
}

fr_status ensure_tmp(fr_batch* b, size_t bytes) {
    if (bytes <= b->tmp_bytes) return FR_OK;
    BCU(cudaStreamSynchronize(b->s));
    cudaFree(b->tmp);
    b->tmp = nullptr;
    b->tmp_bytes = 0;
    BCU(cudaMalloc(&b->tmp, bytes));
    b->tmp_bytes = bytes;
    return FR_OK;
}

void free_batch(fr_batch* b) {
    drop_graph(b);
    for (auto& k : b->bk) cudaFree(k.d_chunks);
    cudaFree(b->arena);
    cudaFree(b->hist_arena);
    cudaFree(b->d_args_sweep);
    cudaFree(b->d_args_grad);
    cudaFree(b->d_red);
    cudaFree(b->d_red0);
    cudaFree(b->d_adam);
    cudaFree(b->d_args_p1);
    cudaFree(b->d_red_map);
    cudaFree(b->d_adam_map);
    cudaFree(b->flags);
    cudaFree(b->tmp);
    if (b->st_host) cudaFreeHost(b->st_host);
    for (int j = 0; j < b->nside; ++j) {
        if (b->side[j]) cudaStreamDestroy(b->side[j]);
        if (b->ev_join[j]) cudaEventDestroy(b->ev_join[j]);
    }
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->s) cudaStreamDestroy(b->s);
}

fr_batch* checked(fr_batch* b, int32_t market, fr_status* st) {
    if (!b) {
        *st = bfail(nullptr, FR_EINVAL, "batch is NULL");
        return nullptr;
    }
    if (market < 0 || market >= b->M) {
        *st = bfail(b, FR_EINVAL, "market %d outside [0, %d)", market, b->M);
        return nullptr;
    }
    return b;
}

}  // namespace

extern "C" {

fr_status fr_batch_create(const fr_config* cfgs, int32_t n_markets, void* stream, fr_batch** out) {
    NvtxRange nvtx_range("fr_batch_create");
    fr_batch* b = nullptr;
    if (!out) return bfail(nullptr, FR_EINVAL, "out is NULL");
    *out = nullptr;
    if (!cfgs || n_markets < 1) return bfail(nullptr, FR_EINVAL, "need cfgs and n_markets >= 1");
    const fr_config& c0 = cfgs[0];
    for (int i = 0; i < n_markets; ++i) {
        const fr_config& c = cfgs[i];
        if (c.n_users < 1 || c.n_items < 1 || c.n_slots < 1 || c.n_slots > c.n_items)
            return bfail(nullptr, FR_EINVAL, "market %d: need n_users >= 1 and 1 <= n_slots <= n_items", i);
        if (c.param != FR_PARAM_ITEM && c.param != FR_PARAM_FULL_C)
            return bfail(nullptr, FR_EINVAL, "market %d: unknown param %d", i, c.param);
        if (c.param != c0.param)
            return bfail(nullptr, FR_EINVAL, "market %d: every market needs market 0's param", i);
        if (c.param == FR_PARAM_FULL_C && c.rel_dtype != FR_F32)
            return bfail(nullptr, FR_EUNSUPPORTED, "market %d: FR_PARAM_FULL_C stores relevance in FP32", i);
        if (c.grad_mode != FR_GRAD_IMPLICIT)
            return bfail(nullptr, FR_EUNSUPPORTED, "market %d: batches differentiate implicitly", i);
        if (c.epsilon != c0.epsilon || c.sinkhorn_iters != c0.sinkhorn_iters ||
            c.warm_start != c0.warm_start || c.optimizer != c0.optimizer || c.lr != c0.lr ||
            c.beta1 != c0.beta1 || c.beta2 != c0.beta2 || c.adam_eps != c0.adam_eps ||
            c.rel_dtype != c0.rel_dtype || c.max_wait_polls != c0.max_wait_polls)
            return bfail(nullptr, FR_EINVAL, "market %d: every field but the sizes must equal market 0's", i);
        for (int j = 0; j < 6; ++j)
            if (c.reserved[j]) return bfail(nullptr, FR_EINVAL, "reserved fields must be zero");
        const int nc = fr_num_cols(c.n_items, c.n_slots);
        P1Variant v1{};
        if (c.param == FR_PARAM_FULL_C) {
            if (!p1_select_batch(nc, c.n_items, &v1))
                return bfail(nullptr, FR_EUNSUPPORTED,
                             "market %d: FR_PARAM_FULL_C needs n_cols <= 64 and n_items within the "
                             "compiled variants (got %d, %d)", i, nc, c.n_items);
        } else if (nc > 32 || warps_at(c.n_items, 8) * 32 > 512) {
            return bfail(nullptr, FR_EUNSUPPORTED,
                         "market %d: batches need n_cols <= 32 and n_items <= 4096 (got %d, %d)", i,
                         nc, c.n_items);
        }
    }
    if (!(c0.epsilon > 0.0) || !std::isfinite(c0.epsilon) || c0.sinkhorn_iters < 1 || !(c0.lr > 0.0) ||
        !(c0.beta1 >= 0.0 && c0.beta1 < 1.0) || !(c0.beta2 >= 0.0 && c0.beta2 < 1.0) ||
        !(c0.adam_eps >= 0.0) || (c0.optimizer != FR_ADAM && c0.optimizer != FR_SGD) ||
        (c0.rel_dtype != FR_F32 && c0.rel_dtype != FR_BF16) || c0.max_wait_polls < -1)
        return bfail(nullptr, FR_EINVAL, "invalid shared configuration");

    b = new fr_batch();
    b->cfg = c0;
    b->p1 = c0.param == FR_PARAM_FULL_C;
    b->M = n_markets;
    b->esz = c0.rel_dtype == FR_BF16 ? 2 : 4;
    b->user = (cudaStream_t)stream;
    auto bail = [&](fr_status st) {
        g_batch_create_error = b->err;
        free_batch(b);
        delete b;
        return st;
    };
#define BCC(call)                                                                                \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return bail(bfail(b, e_ == cudaErrorMemoryAllocation ? FR_ENOMEM : FR_ECUDA, "%s: %s", \
                              #call, cudaGetErrorString(e_)));                                   \
    } while (0)
    BCC(cudaGetDevice(&b->device));
    BCC(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device));
    BCC(cudaDeviceGetAttribute(&b->max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device));
    BCC(cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking));
    BCC(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    BCC(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    BCC(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));

    // markets and buckets
    b->mk.resize(n_markets);
    for (int i = 0; i < n_markets; ++i) {
        BMarket& m = b->mk[i];
        m.U = cfgs[i].n_users;
        m.I = cfgs[i].n_items;
        m.K = cfgs[i].n_slots;
        m.nc = fr_num_cols(m.I, m.K);
        m.ld = (m.I + 7) / 8 * 8;
        m.rows = (m.U + kCpcMin - 1) / kCpcMin;
        int kb = -1;
        if (b->p1) {  // free costs: one bucket per kernel variant (columns, rows, tile stride)
            P1Variant v{};
            p1_select_batch(m.nc, m.I, &v);
            for (size_t j = 0; j < b->bk.size(); ++j) {
                const P1Variant& w = b->bk[j].var1;
                if (w.ncb == v.ncb && w.rows == v.rows && w.exact == v.exact &&
                    w.tile_stride == v.tile_stride)
                    kb = (int)j;
            }
            if (kb < 0) {
                BBucket k;
                k.ncb = v.ncb;
                k.exact = v.exact;
                k.var1 = v;
                b->bk.push_back(k);
                kb = (int)b->bk.size() - 1;
            }
            BBucket& k = b->bk[kb];
            k.var1.threads = std::max(k.var1.threads, v.threads);  // the bucket's largest market
            k.markets.push_back(i);
            k.I_max = std::max(k.I_max, m.I);
            k.ld_max = std::max(k.ld_max, m.ld);
            m.bucket = kb;
            continue;
        }
        const int ncb = ncb_of(m.nc), w8 = warps_at(m.I, 8);
        for (size_t j = 0; j < b->bk.size(); ++j)
            if (b->bk[j].ncb == ncb && b->bk[j].warps8 == w8) kb = (int)j;
        if (kb < 0) {
            BBucket k;
            k.ncb = ncb;
            k.exact = ncb == 6 || ncb == 11 || ncb == 21;  // kernels with 16 / 24 rows per thread
            k.warps8 = w8;
            b->bk.push_back(k);
            kb = (int)b->bk.size() - 1;
        }
        BBucket& k = b->bk[kb];
        k.markets.push_back(i);
        k.I_max = std::max(k.I_max, m.I);
        k.ld_max = std::max(k.ld_max, m.ld);
        m.bucket = kb;
    }
    b->nside = std::min<int>(kMaxSide, (int)b->bk.size());
    for (int j = 0; j < b->nside; ++j) {
        BCC(cudaStreamCreateWithFlags(&b->side[j], cudaStreamNonBlocking));
        BCC(cudaEventCreateWithFlags(&b->ev_join[j], cudaEventDisableTiming));
    }

    // one arena for every per-market buffer (256-byte aligned pieces)
    size_t total = 0;
    auto piece = [&](size_t bytes) {
        const size_t o = total;
        total += (bytes + 255) / 256 * 256;
        return o;
    };
    struct Off { size_t r, th, m1, m2, w, gL, gP, e, lb, om, part, gpart, imp, blk, ad, gn2, st,
                 C, c1, c2; };
    std::vector<Off> off(n_markets);
    const size_t per_item = b->p1 ? 0 : 1, per_cell = b->p1 ? 1 : 0;
    for (int i = 0; i < n_markets; ++i) {
        const BMarket& m = b->mk[i];
        const size_t ld = m.ld, un = (size_t)m.U * m.nc;
        Off& o = off[i];
        o.r = piece((size_t)m.U * ld * b->esz);
        o.th = piece(4 * ld * per_item); o.m1 = piece(4 * ld * per_item);
        o.m2 = piece(4 * ld * per_item); o.w = piece(4 * ld * per_item);
        o.C = piece(4 * un * ld * per_cell); o.c1 = piece(4 * un * ld * per_cell);
        o.c2 = piece(4 * un * ld * per_cell);
        o.gL = piece(4 * un); o.gP = piece(4 * un);
        o.e = piece(4 * (size_t)m.nc); o.lb = piece(4 * (size_t)m.nc); o.om = piece(4 * ld);
        o.part = piece(4 * (size_t)m.rows * ld); o.gpart = piece(4 * (size_t)m.rows * ld * per_item);
        o.imp = piece(8 * ld); o.blk = piece(16 * (size_t)reduce_blocks(m.I));
        o.ad = piece(8 * (size_t)p2_adam_blocks(m.I) * per_item);
        o.gn2 = piece(8 * (b->p1 ? (size_t)m.rows : 1));  // free costs: one partial per chunk row
        o.st = piece(sizeof(DevState));
    }
    BCC(cudaMalloc(&b->arena, total));
    BCC(cudaMemset(b->arena, 0, total));
    unsigned char* base = static_cast<unsigned char*>(b->arena);
    for (int i = 0; i < n_markets; ++i) {
        BMarket& m = b->mk[i];
        const Off& o = off[i];
        m.r = base + o.r;
        m.theta = (float*)(base + o.th); m.tm1 = (float*)(base + o.m1); m.tm2 = (float*)(base + o.m2);
        m.w = (float*)(base + o.w); m.gL = (float*)(base + o.gL); m.gP = (float*)(base + o.gP);
        m.e = (float*)(base + o.e); m.invb = (float*)(base + o.lb); m.omega = (float*)(base + o.om);
        m.part = (float*)(base + o.part); m.gpart = (float*)(base + o.gpart);
        m.imp = (double*)(base + o.imp); m.blk = (double*)(base + o.blk);
        m.ad_blk = (double*)(base + o.ad); m.gn2 = (double*)(base + o.gn2);
        m.st = (DevState*)(base + o.st);
        if (b->p1) {
            m.C = (float*)(base + o.C); m.m1 = (float*)(base + o.c1); m.m2 = (float*)(base + o.c2);
        }
    }
    BCC(cudaMalloc(&b->d_args_sweep, sizeof(P2Args) * n_markets));
    BCC(cudaMalloc(&b->d_args_grad, sizeof(P2Args) * n_markets));
    BCC(cudaMalloc(&b->d_red, sizeof(ReduceArgs) * n_markets));
    BCC(cudaMalloc(&b->d_red0, sizeof(ReduceArgs) * n_markets));
    BCC(cudaMalloc(&b->d_adam, sizeof(P2AdamArgs) * n_markets));
    if (b->p1) BCC(cudaMalloc(&b->d_args_p1, sizeof(P1Args) * n_markets));
    BCC(cudaMalloc(&b->flags, sizeof(int) * 4));
    BCC(cudaMallocHost(&b->st_host, sizeof(DevState) * n_markets));
    std::vector<int2> rmap, amap;
    for (int i = 0; i < n_markets; ++i) {
        for (int j = 0; j < reduce_blocks(b->mk[i].I); ++j) rmap.push_back(make_int2(i, j));
        if (!b->p1)
            for (int j = 0; j < p2_adam_blocks(b->mk[i].I); ++j) amap.push_back(make_int2(i, j));
    }
    b->n_red_blocks = (int)rmap.size();
    b->n_adam_blocks = (int)amap.size();
    BCC(cudaMalloc(&b->d_red_map, sizeof(int2) * rmap.size()));
    BCC(cudaMalloc(&b->d_adam_map, sizeof(int2) * std::max<size_t>(amap.size(), 1)));
    BCC(cudaMemcpy(b->d_red_map, rmap.data(), sizeof(int2) * rmap.size(), cudaMemcpyHostToDevice));
    if (!amap.empty())
        BCC(cudaMemcpy(b->d_adam_map, amap.data(), sizeof(int2) * amap.size(), cudaMemcpyHostToDevice));
#undef BCC
    for (auto& k : b->bk) {
        fr_status st = b->p1 ? configure_bucket_p1(b, k, kCpcMin) : configure_bucket(b, k, 8, kCpcMin);
        if (st != FR_OK) return bail(st);
    }
    fr_status st = ensure_hist(b, 64);  // also uploads the argument tables
    if (st != FR_OK) return bail(st);
    if ((st = zero_state(b)) != FR_OK) return bail(st);
    *out = b;
    return FR_OK;
}

fr_status fr_batch_destroy(fr_batch* b) {
    if (!b) return FR_OK;
    cudaStreamSynchronize(b->s);
    free_batch(b);
    delete b;
    return FR_OK;
}

fr_status fr_batch_reset(fr_batch* b) {
    if (!b) return bfail(nullptr, FR_EINVAL, "batch is NULL");
    BJoin j(b);
    return zero_state(b);
}

fr_status fr_batch_set_relevance(fr_batch* b, int32_t market, const void* r, int32_t dtype, int64_t ld,
                                 int32_t on_device) {
    NvtxRange nvtx_range("fr_batch_set_relevance");
    fr_status st = FR_OK;
    if (!checked(b, market, &st)) return st;
    BMarket& m = b->mk[market];
    if (!r) return bfail(b, FR_EINVAL, "r is NULL");
    if (dtype != FR_F32 && dtype != FR_F64 && dtype != FR_BF16)
        return bfail(b, FR_EINVAL, "unknown dtype %d", dtype);
    if (ld < m.I) return bfail(b, FR_EINVAL, "ld %lld < n_items %d", (long long)ld, m.I);
    BJoin j(b);
    const size_t esz = dtype == FR_F64 ? 8 : dtype == FR_F32 ? 4 : 2;
    const void* src = r;
    int64_t lds = ld;
    if (!on_device) {
        if ((st = ensure_tmp(b, esz * (size_t)m.U * m.I)) != FR_OK) return st;
        BCU(cudaMemcpy2DAsync(b->tmp, esz * m.I, r, esz * ld, esz * m.I, m.U, cudaMemcpyHostToDevice, b->s));
        src = b->tmp;
        lds = m.I;
    }
    BCU(launch_relevance_import(src, dtype, lds, m.r, b->esz == 2, m.U, m.I, m.ld, b->s));
    BCU(cudaMemsetAsync(b->flags, 0, sizeof(int) * 4, b->s));
    BCU(launch_relevance_check(m.r, b->esz == 2, m.U, m.I, m.ld, b->flags, b->s));
    b->launches += 2;
    int hf[4];
    BCU(cudaMemcpyAsync(hf, b->flags, sizeof hf, cudaMemcpyDeviceToHost, b->s));
    BCU(cudaStreamSynchronize(b->s));
    if (hf[0]) return bfail(b, FR_EINVAL, "market %d: relevance must be finite and >= 0", market);
    if (hf[1])
        return bfail(b, FR_EINVAL, "market %d: %d items have no positive relevance", market, hf[1]);
    m.have_r = true;
    b->fresh = false;
    return FR_OK;
}

fr_status fr_batch_set_exposure(fr_batch* b, int32_t market, const double* e, int32_t K) {
    fr_status st = FR_OK;
    if (!checked(b, market, &st)) return st;
    BMarket& m = b->mk[market];
    if (!e) return bfail(b, FR_EINVAL, "e is NULL");
    if (K != m.K) return bfail(b, FR_EINVAL, "market %d: K %d != n_slots %d", market, K, m.K);
    std::vector<float> ep(m.nc, 0.f), lb(m.nc, 1.f);  // lb: 1 / b_k
    float emax = 0.f;
    for (int k = 0; k < K; ++k) {
        if (!(e[k] > 0.0) || !std::isfinite(e[k]))
            return bfail(b, FR_EINVAL, "market %d: exposure e[%d] must be positive and finite", market, k);
        ep[k] = (float)e[k];
        emax = std::max(emax, ep[k]);
    }
    if (m.nc > K) lb[K] = (float)(1.0 / (double)(m.I - K));  // dummy mass |I| - K
    BJoin j(b);
    BCU(cudaMemcpyAsync(m.e, ep.data(), sizeof(float) * m.nc, cudaMemcpyHostToDevice, b->s));
    BCU(cudaMemcpyAsync(m.invb, lb.data(), sizeof(float) * m.nc, cudaMemcpyHostToDevice, b->s));
    BCU(cudaStreamSynchronize(b->s));
    if (m.emax != emax) {  // the sweep arguments carry e_max
        m.emax = emax;
        if ((st = upload_tables(b)) != FR_OK) return st;
    }
    m.have_e = true;
    b->fresh = false;
    return FR_OK;
}

fr_status fr_batch_autotune(fr_batch* b) {
    NvtxRange nvtx_range("fr_batch_autotune");
    if (!b) return bfail(nullptr, FR_EINVAL, "batch is NULL");
    for (int i = 0; i < b->M; ++i)
        if (!b->mk[i].have_r || !b->mk[i].have_e)
            return bfail(b, FR_ESTATE, "market %d: set relevance and exposure first", i);
    BJoin j(b);
    return autotune(b);
}

fr_status fr_batch_step(fr_batch* b, int32_t n_steps, double* nsw_trace) {
    NvtxRange nvtx_range("fr_batch_step");
    if (!b) return bfail(nullptr, FR_EINVAL, "batch is NULL");
    if (n_steps < 0) return bfail(b, FR_EINVAL, "n_steps < 0");
    BJoin j(b);
    fr_status st = ensure_ready(b);
    if (st != FR_OK) return st;
    if ((st = ensure_hist(b, n_steps)) != FR_OK) return st;
    if ((st = set_run_states(b)) != FR_OK) return st;
    int done = 0;
    if (n_steps >= kBatchChunk && (st = ensure_graph(b)) != FR_OK) return st;
    while (n_steps - done >= kBatchChunk) {
        BCU(cudaGraphLaunch(b->chunk_exec, b->s));
        b->launches += (int64_t)kernels_per_step(b) * kBatchChunk;
        done += kBatchChunk;
    }
    for (; done < n_steps; ++done)
        if ((st = launch_step(b)) != FR_OK) return st;
    if ((st = read_states(b)) != FR_OK) return st;
    if (nsw_trace && n_steps > 0) {
        std::vector<double> h(n_steps);
        for (int i = 0; i < b->M; ++i) {
            BCU(cudaMemcpyAsync(h.data(), b->mk[i].F_hist, sizeof(double) * n_steps,
                                cudaMemcpyDeviceToHost, b->s));
            BCU(cudaStreamSynchronize(b->s));
            for (int t = 0; t < n_steps; ++t) nsw_trace[(size_t)t * b->M + i] = h[t];
        }
    }
    return FR_OK;
}

fr_status fr_batch_impacts(fr_batch* b, int32_t market, double* imp_out, double* utility_out,
                           double* nsw_out) {
    NvtxRange nvtx_range("fr_batch_impacts");
    fr_status st = FR_OK;
    if (!checked(b, market, &st)) return st;
    BJoin j(b);
    if ((st = ensure_ready(b)) != FR_OK) return st;
    const BMarket& m = b->mk[market];
    if (imp_out)
        BCU(cudaMemcpyAsync(imp_out, m.imp, sizeof(double) * m.I, cudaMemcpyDeviceToHost, b->s));
    if ((st = read_states(b)) != FR_OK) return st;
    if (utility_out) *utility_out = b->st_host[market].utility;
    if (nsw_out) *nsw_out = b->st_host[market].F;
    return FR_OK;
}

fr_status fr_batch_policy(fr_batch* b, int32_t market, int32_t u0, int32_t n_u, float* x_out,
                          int32_t on_device) {
    NvtxRange nvtx_range("fr_batch_policy");
    fr_status st = FR_OK;
    if (!checked(b, market, &st)) return st;
    const BMarket& m = b->mk[market];
    if (u0 < 0 || n_u < 0 || (int64_t)u0 + n_u > m.U)
        return bfail(b, FR_EINVAL, "consumer range [%d, %d) outside [0, %d)", u0, u0 + n_u, m.U);
    if (!x_out && n_u > 0) return bfail(b, FR_EINVAL, "x_out is NULL");
    BJoin j(b);
    if ((st = ensure_ready(b)) != FR_OK) return st;
    const size_t bytes = sizeof(float) * (size_t)n_u * m.I * m.nc;
    float* dst = x_out;
    if (!on_device) {
        if ((st = ensure_tmp(b, bytes)) != FR_OK) return st;
        dst = b->tmp;
    }
    if (b->p1)
        BCU(launch_policy(market_args_p1(b, m), u0, n_u, dst, b->s));
    else
        BCU(launch_p2_policy(market_args(b, m, m.part), u0, n_u, dst, b->s));
    b->launches += n_u > 0;
    if (!on_device && n_u > 0) BCU(cudaMemcpyAsync(x_out, dst, bytes, cudaMemcpyDeviceToHost, b->s));
    BCU(cudaStreamSynchronize(b->s));
    return FR_OK;
}

fr_status fr_batch_get_theta(fr_batch* b, int32_t market, float* theta_out) {
    fr_status st = FR_OK;
    if (!checked(b, market, &st)) return st;
    if (!theta_out) return bfail(b, FR_EINVAL, "theta_out is NULL");
    if (b->p1) return bfail(b, FR_EINVAL, "free-cost markets have no per-item variables");
    BJoin j(b);
    const BMarket& m = b->mk[market];
    BCU(cudaMemcpyAsync(theta_out, m.theta, sizeof(float) * m.I, cudaMemcpyDeviceToHost, b->s));
    BCU(cudaStreamSynchronize(b->s));
    return FR_OK;
}

fr_status fr_batch_tuning(const fr_batch* b, int32_t* n_buckets, int32_t* table, int32_t cap) {
    if (!b) return bfail(nullptr, FR_EINVAL, "batch is NULL");
    if (n_buckets) *n_buckets = (int32_t)b->bk.size();
    if (table)
        for (int i = 0; i < (int)b->bk.size() && i < cap; ++i) {
            const BBucket& k = b->bk[i];
            int32_t* t = table + 6 * i;
            t[0] = k.ncb;
            t[1] = (int32_t)k.markets.size();
            t[2] = k.I_max;
            t[3] = k.R;
            t[4] = b->p1 ? k.var1.threads : k.var.threads;
            t[5] = k.cpc;
        }
    return FR_OK;
}

const char* fr_batch_last_error(const fr_batch* b) {
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}

int64_t fr_batch_launch_count(const fr_batch* b) { return b ? b->launches : 0; }

}  // extern "C"
