// fr_internal.h -- structures shared by the libfairrank translation units (host + device).
//
// Device layout of one problem (all owned by the context):
//   C, m1, m2   float [U][nc][ld]  costs and Adam moments, k-major per consumer so that a thread
//                                  owning consecutive items i reads/writes them with coalesced
//                                  vector accesses (ld = n_items rounded up to a multiple of 8,
//                                  padding rows are zero and never enter any sum)
//   r           float [U][ld]      relevance r(u,i)
//   gL, gP      float [U][nc]      column potentials in log2 units, g' = g / (eps ln 2): gL is the
//                                  last solve's g^(L) (the warm start), gP its g^(L-1) (the
//                                  potentials the emitted policy was formed with)
//   part        float [G][ld]      per-CTA partial impacts sum_u r(u,i) v(u,i) of the last sweep
//   gn2_part    double [G]         per-CTA partial squared gradient norms
//   imp         double [ld]        Imp_i (Eq. 4) after the cross-CTA reduction
//   omega       float [ld]         dF/dImp_i = 1/Imp_i for the next gradient
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "fairrank.h"

namespace fr {

// NVTX range over a public entry point: names the call on a profiler's timeline (header-only NVTX
// 3; without a tool attached the push / pop return at once).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};


// Device-resident step state: read and written by the kernels so that captured CUDA graphs can
// be replayed without changing kernel arguments.
struct DevState {
    long long t;          // Adam steps applied
    int hist_idx;         // next slot of the F / gradient-norm history
    int stop;             // set by the reduction when a step's gradient norm <= thresh
    int err;              // bit 0: non-positive or non-finite impact; bit 1: non-finite gradient
    int steps_done;       // steps applied since the host last cleared it
    unsigned int counter; // last-block-done counter of the reduction (returns to 0)
    int max_steps;        // > 0: the reduction raises stop once steps_done reaches it
    unsigned long long log_solves;  // tile-sweep solves that finished in the log form
    unsigned long long cta_ns;      // free-cost update step: CTA 0's duration per consumer (ns) in
                                    // the last launch (0 before the first), for the stagger below
    double F, utility, gnorm;
    double thresh;        // < 0: never stop
};

enum Mode { MODE_SWEEP = 0, MODE_UPDATE_SWEEP = 1, MODE_GRAD = 2 };

struct P1Args {
    int U, I, K, nc, ld, L, G;
    float* C;
    float* m1;
    float* m2;
    float* gL;
    float* gP;
    const float* r;
    const float* e;       // [nc] exposure, dummy = 0
    const float* invb;    // [nc] 1 / b_k of the column marginals
    const float* omega;   // [ld]
    float* part;          // [G][ld]
    double* gn2_part;     // [G]
    DevState* st;
    float* dC;            // MODE_GRAD: dF/dC, [U][I][nc] (public layout)
    float* dr;            // MODE_GRAD: dF/dr, [U][I] (nullable)
    float inv_eps_ln2;    // 1 / (eps ln 2)
    float inv_eps;
    float lr, beta1, beta2, adam_eps;
    int optimizer;        // 0 Adam, 1 SGD
    int warm;
    unsigned max_polls;   // bounded waits: polls before a wait gives up (0: expires at once)
    float* g0;            // unrolled gradient: [U][nc] log2-unit potentials each solve started
                          // from, stored by the sweeps when non-null
    int ce, nck;          // unrolled gradient: checkpoint interval and count ceil(L / ce)
    float* gall;          // with a checkpoint every iteration: g' at the start of every iteration
    float* csall;         // and its column sums, [U][L][nc] each, stored by the sweeps (nullable;
                          // the unrolled gradient then does no forward re-runs)
};

struct ReduceArgs {
    int I, ld, G, U;
    int Ggn;              // number of squared-gradient-norm partials (G for the free-cost path)
    const float* part;
    const double* gn2_part;
    double* imp;
    float* omega;
    double* blk;          // [nblocks][2] partial (sum log Imp, sum Imp)
    DevState* st;
    double* F_hist;
    double* gn_hist;
    int hist_cap;
    int after_update;     // 1 if the sweep followed an optimiser update
    int nblk;             // batched launches: reduction blocks of this problem
};

// ---- per-item parametrisation c_uik = -r(u,i) e_k exp(theta_i) ----------------------------------
struct P2Args {
    int U, I, K, nc, ld, L, G;
    const void* r;        // [U][ld] relevance, float or bfloat16 (r_bf16)
    int r_bf16;
    const float* w;       // [ld] exp(theta)
    const float* e;       // [nc] exposure, dummy = 0
    const float* invb;    // [nc] 1 / b_k
    float emax;           // max_k e_k
    float* gL;            // [U][nc] log2-unit potentials (re-referenced to the last column)
    float* gP;
    float* part;          // [G][ld] per-CTA impact partials (sweep) or dL/dtheta partials (grad)
    const float* omega;   // [ld] dL/dImp_i (grad)
    float* dr;            // grad: dL/dr [U][I] (nullable)
    DevState* st;
    float inv_eps_ln2, inv_eps;
    int warm;
    float* ck;            // unrolled gradient: column-potential checkpoints [U][nck][nc] (nullable)
    int ce, nck;          // checkpoint interval (iterations) and count ceil(L / ce)
    float* csk;           // with a checkpoint every iteration: the column sums cs^(l+1) of every
                          // iteration l [U][L][nc], so the adjoint skips its forward re-runs
                          // (nullable)
    unsigned max_polls;   // bounded waits: polls before a wait gives up (0: expires at once)
};

// Batched markets: a launch processes a list of chunks, each a range of consumers of one market
// with its own row of the market's partial buffer (mk[market].part + row * ld).
struct P2Chunk {
    int market, u0, u1, row;
};

struct P2Batch {
    const P2Args* mk;     // device array of per-market arguments (nullptr: single-market launch)
    const P2Chunk* ch;    // device array of this launch's chunks
    int n_chunks;
    int ld_max;           // largest ld of the chunks' markets (shared-memory layout)
    int esz;              // bytes per stored relevance value (shared by all markets)
};

struct P2Variant {
    int ncb, rows, exact, threads;
    const void* sweep;
    const void* grad;
    const void* sweep_b;  // batched-market forms of sweep / grad (argument: P2Batch)
    const void* grad_b;
    const void* adj;      // unrolled-gradient (adjoint) kernel, CTA of adj_threads (p2_select_adj)
    int adj_threads;
};

// dL/dtheta from the per-CTA partials (FP64, fixed order), its squared norm, and optionally the
// optimiser step on theta (w = exp(theta) refreshed).
struct P2AdamArgs {
    int I, ld, G;
    const float* part;    // [G][ld]
    float* theta;
    float* m1;
    float* m2;
    float* w;
    float* dtheta_out;    // nullable: dL/dtheta as float [I]
    double* gn2_out;      // squared norm (one partial for the reduction kernel)
    double* blk;          // [nblocks] per-block partial squared norms
    DevState* st;
    float lr, beta1, beta2, adam_eps;
    int optimizer;        // 0 Adam, 1 SGD
    int apply;            // 0: gradient only
    int nblk;             // batched launches: update blocks of this problem
};

// Polls of a bounded device-side wait by default (fr_config.max_wait_polls = 0), and the polls of
// the drain that follows an expired wait (a kernel never leaves with its own copies in flight).
constexpr unsigned kDefaultPolls = 1u << 26;
// fr_config.max_wait_polls -> polls per wait
inline unsigned polls_of(int32_t max_wait_polls) {
    return max_wait_polls == 0 ? kDefaultPolls : max_wait_polls < 0 ? 0u : (unsigned)max_wait_polls;
}

// Raises a kernel's dynamic shared-memory limit to at least `bytes` (never lowers it: the limit is
// per function, shared by every context that launches it). Serialised by a process-wide lock.
cudaError_t raise_smem_limit(const void* fn, size_t bytes);

bool p2_select(int nc, int I, P2Variant* out);
size_t p2_sweep_smem(const P2Variant& v, int nc, int ld, int esz);
size_t p2_grad_smem(const P2Variant& v, int nc, int ld, int esz);
cudaError_t p2_launch_sweep(const P2Variant& v, const P2Args& a, cudaStream_t s);
cudaError_t p2_launch_grad(const P2Variant& v, const P2Args& a, cudaStream_t s);
// batched launches: grid G, shared memory for ld_max (all markets of the launch share ncb)
size_t p2_sweep_smem_batch(const P2Variant& v, int ld_max, int esz);
size_t p2_grad_smem_batch(const P2Variant& v, int ld_max, int esz);
cudaError_t p2_launch_sweep_batch(const P2Variant& v, const P2Batch& bt, int G, cudaStream_t s);
cudaError_t p2_launch_grad_batch(const P2Variant& v, const P2Batch& bt, int G, cudaStream_t s);
bool p2_select_adj(int nc, int I, P2Variant* v);  // sets adj / adj_threads
bool p2_adj_k21(int R, int threads, P2Variant* v);
bool p2_adj_k11_k6(int nc, int R, int threads, P2Variant* v);
bool p2_adj_generic(int ncb, int threads, P2Variant* v);
size_t p2_adj_smem(const P2Variant& v, int nc, int ld, int esz, int ce);
cudaError_t p2_launch_adj(const P2Variant& v, const P2Args& a, cudaStream_t s);
cudaError_t p2_launch_adam(const P2AdamArgs& a, cudaStream_t s);
// batched markets: block j works on block bmap[j].y of market bmap[j].x (device arrays)
cudaError_t p2_launch_adam_batch(const P2AdamArgs* aa, const int2* bmap, int nblocks, cudaStream_t s);
cudaError_t launch_exp_theta(const float* theta, float* w, int I, int ld, cudaStream_t s);
cudaError_t launch_p2_policy(const P2Args& a, int u0, int n_u, float* x, cudaStream_t s);
int p2_adam_blocks(int I);
bool p2_variant_k21(int R, int threads, P2Variant* out);
bool p2_variant_k11(int R, int threads, P2Variant* out);
bool p2_variant_k6(int R, int threads, P2Variant* out);
bool p2_variant_generic(int ncb, int threads, P2Variant* out);

// Launchers (return cudaError_t of the launch). `variant` is resolved by p1_select.
struct P1Variant {
    int ncb, rows, exact;
    int tile_stride;      // 0: register sweep; else the Sinkhorn phase reads its costs from the
                          // resident shared tile, whose columns are tile_stride floats apart
    int threads;          // CTA size
    size_t smem;          // dynamic shared memory (bytes) of the largest mode
    const void* fn[3];    // kernels by Mode
    const void* fn_rec;   // MODE_SWEEP that also records g' and the column sums of every iteration
                          // (P1Args::gall / csall), for the unrolled gradient
    const void* fb[2];    // batched-market kernels (argument: P1Batch) for MODE_SWEEP and
                          // MODE_UPDATE_SWEEP; set by p1_select_batch only
};

// Batched free-cost markets: a launch walks a chunk list (P2Chunk: market, consumer range, partial
// row); every market's arguments are in a device table. All markets of a launch share the kernel
// variant; the shared-memory layout is the variant's at ld_max.
struct P1Batch {
    const P1Args* mk;
    const P2Chunk* ch;
    int n_chunks;
    int ld_max;
};

bool p1_select(int nc, int I, P1Variant* out);
// The same variant table as p1_select, with fb set (and fn left null).
bool p1_select_batch(int nc, int I, P1Variant* out);
size_t p1_smem_bytes_batch(const P1Variant& v, int mode, int ld_max);
cudaError_t p1_launch_batch(const P1Variant& v, int mode, const P1Batch& bt, int G, cudaStream_t s);

// Unrolled gradient of the free-cost parametrisation (fr_p1_adj.cu): fn[0] writes dL/dC and
// dL/dr, fn[1] applies the optimiser step to C (mode = 0 / 1).
struct P1AdjVariant {
    int ncb, rows, exact, threads;
    const void* fn[2];
};
bool p1_select_adj(int nc, int I, P1AdjVariant* out);
size_t p1_adj_smem(const P1AdjVariant& v, int nc, int ld, int ce, int nck);
cudaError_t p1_launch_adj(const P1AdjVariant& v, int mode, const P1Args& a, int G, cudaStream_t s);
cudaError_t p1_launch(const P1Variant& v, int mode, const P1Args& a, cudaStream_t s);
size_t p1_smem_bytes(const P1Variant& v, int mode, int nc, int ld);
cudaError_t reduce_launch(const ReduceArgs& a, cudaStream_t s);
cudaError_t reduce_launch_batch(const ReduceArgs* ra, const int2* bmap, int nblocks, cudaStream_t s);
int reduce_blocks(int I);

cudaError_t launch_pack_ikn_to_kni(const float* src, float* dst, int U, int I, int nc, int ld,
                                   float scale, cudaStream_t s);
cudaError_t launch_unpack_kni_to_ikn(const float* src, float* dst, int U, int I, int nc, int ld,
                                     float scale, cudaStream_t s);
cudaError_t launch_scale(const float* src, float* dst, long long n, float scale, cudaStream_t s);
// relevance [U][I] (row stride ld_src, dtype FR_F32 | FR_F64 | FR_BF16) -> [U][ld] stored as
// float or bfloat16 (dst_bf16, round to nearest even), padding zero
cudaError_t launch_relevance_import(const void* src, int dtype, long long ld_src, void* dst,
                                    int dst_bf16, int U, int I, int ld, cudaStream_t s);
cudaError_t launch_relevance_check(const void* r, int r_bf16, int U, int I, int ld, int* flags,
                                   cudaStream_t s);
cudaError_t launch_policy(const P1Args& a, int u0, int n_u, float* x_out, cudaStream_t s);
cudaError_t launch_ex2_bench(float* sink, int blocks, int threads, int iters, cudaStream_t s);
// kind 0 / 1: shared-memory loads of 8 / 16 bytes; 2 / 3: scalar / packed FP32 FMA. clk[0..1]: SM
// cycles and nanoseconds of block 0's loop.
// self-check of log2_near1 over every float of its short path (fr_common.cu): out[3] unsigned,
// zeroed by the caller: max relative errors of log2_near1 and log2f as float bits, misses at y = 1
cudaError_t launch_log2_check(unsigned* out, int blocks, cudaStream_t s);
cudaError_t launch_peak_bench(int kind, float* sink, int blocks, int threads, int iters,
                              unsigned long long* clk, cudaStream_t s);
// Body end of fr_solve's device-side while loop: ctl[0] counts body iterations, ctl[1] caps them;
// sets the loop's condition to continue while no stop / error flag is raised and the cap is not hit.
cudaError_t launch_solve_cond(const DevState* st, int* ctl, cudaGraphConditionalHandle h,
                              cudaStream_t s);

// evaluation metrics (fr_metrics.cu): v_ui = sum_{k<K} e_k x_uik into V [U][ld]; then the envy
// contraction E = R^T V with its row-max epilogue, column sums of r and the ratio tests. out[3]:
// mean max envy, % better off, % worse off. Scratch: rmax [envy_tc_tiles(I)][ld] floats, diag [ld]
// floats, ru [ld] doubles, ru_part [colsum_chunks()][ld] doubles.
// The contraction runs on the tensor cores (fr_envy_tc.cu: 128 x 256-item tiles, three TF32
// products; an expired bounded wait sets bit 4 of *err); rmax holds envy_tc_col_tiles(I) rows, at
// most envy_tc_tiles(I).
int envy_tc_tiles(int I);      // 128-item row tiles
int envy_tc_col_tiles(int I);  // 256-item column tiles
size_t envy_tc_smem();
// scratch of the TF32 planes of R and V (16-byte aligned), written by launch_envy_tc
size_t envy_tc_plane_bytes(int U, int I);
cudaError_t launch_v_p1(const P1Args& a, float* V, cudaStream_t s);
cudaError_t launch_v_p2(const P2Args& a, float* V, cudaStream_t s);
cudaError_t launch_envy_tc(const void* r, int r_bf16, const float* V, int U, int I, int ld,
                           float* rmax, float* diag, int* err, unsigned max_polls, void* planes,
                           cudaStream_t s);
cudaError_t launch_envy(const void* r, int r_bf16, const float* V, int U, int I, int ld,
                        const double* imp, double esum, float* rmax, float* diag, double* ru,
                        double* ru_part, double* out, double* env_item /* nullable, [I] */,
                        int* err, unsigned max_polls, void* planes, cudaStream_t s);
int colsum_chunks();  // FP64 partials [colsum_chunks()][ld] of the column sums of r (ru_part)
// Frank-Wolfe certificate (fr_metrics.cu): one of a1 / a2 non-null (the policy's form); G CTAs
// (cert_grid), per-CTA partials gap_part [G] doubles and res_part [G] floats; out[0] = gap,
// out[1] = column residual.
int cert_grid(int U, int sms);
cudaError_t launch_certificate(const P1Args* a1, const P2Args* a2, const double* imp, int nc, int I,
                               int G, double* gap_part, float* res_part, double* out, cudaStream_t s);

}  // namespace fr
