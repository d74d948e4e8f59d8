// fr_p1.cuh -- kernels of the free-cost parametrisation (Problem (8): one cost c_uik per cell),
// instantiated by fr_p1.cu (the variant table) and fr_p1_k21.cu (21 columns).
//
// One persistent CTA processes consumers u = blockIdx.x, blockIdx.x + G, ... (Algorithm 1's
// parallel loop over consumers). Each consumer's cost tile is bulk-copied (TMA) into shared
// memory: in the register sweep one consumer ahead (with the relevance row), while the previous
// consumer's Sinkhorn iterations run; in the tile sweep, whose solve keeps reading the tile, right
// after the previous solve, from L2 where that solve prefetched it.
//
// Sinkhorn (Problem (7)) runs as one fused pass per iteration, in log2 units
// c' = c / (eps ln 2), g' = g / (eps ln 2):
//   p_ik = 2^(g'_k - c~_ik),  S_i = sum_k p_ik,  x_ik = p_ik / S_i       (row update, Eq. 1)
//   cs_k = sum_i x_ik,        g'_k += log2 b_k - log2 cs_k               (column update, Eq. 2)
// which equals the textbook two-pass update (f_i = -eps LSE_k, g_k = eps log b_k - eps LSE_i)
// algebraically. c~_ik = c'_ik + shift_i carries a per-row shift fixed at the start of the solve
// (the row max), so 2^(.) stays in range without a max pass per iteration. In the register sweep
// a thread owns R consecutive items (rows) and keeps their costs in registers for the whole solve;
// in the tile sweep (tile_sweep below) it owns R / 2 pairs of rows and reads them from the
// resident shared tile every iteration. Both sweeps (the register sweep up to 11 columns) hold
// the row-shifted kernel in its exponential form, E_ik = 2^(g0_k - c~_ik) with g0 the potentials
// at the start of the solve, and form p_ik = E_ik G_k with G_k = 2^(g'_k - g0_k): one multiply
// per cell and one exp2 per column and iteration. While the potentials stay within TS_DRIFT of g0
// this is the same iteration up to FP32 rounding; beyond that (and in the wider register sweeps
// throughout) they use the log form, one exp2 per cell, re-shifting exactly a row whose S_i leaves
// [2^-64, 2^64].
//
// Inner loop: two rows at a time in packed f32x2 arithmetic (one instruction per pair of cells).
// Column sums: per-warp reduce-scatter by shuffles, one
// __syncthreads per iteration on double-buffered partials, after which every warp sums the
// per-warp partials of its lanes' columns in the same fixed order and updates its own copy of the
// column potentials (so no second barrier is needed and every warp holds identical g').
//
// The last iteration emits x (the policy right after the last row update, rows sum to 1) and adds
// r(u,i) * sum_{k<K} e_k x_ik into impact partials (Eq. 4) that accumulate over the CTA's
// consumers in part[blockIdx][i] (per-thread registers written once per launch in the register
// sweep, the partial row itself in the tile sweep); the reduction kernel combines them across CTAs
// in a fixed order.
//
// MODE_UPDATE_SWEEP first takes the gradient step of Algorithm 1 for the consumer, working from
// the shared-memory tile with compact loops (the code runs once per consumer, so it is kept small
// for the instruction cache): it re-forms the previous policy from C and g^(L-1), computes dF/dC
// by implicit differentiation of the optimality conditions of Problem (7),
//   h_i = sum_k x_ik G_ik, q_k = sum_i x_ik G_ik, (diag(cs) - X^T X) beta = q - X^T h (beta_last = 0),
//   alpha_i = h_i - sum_k x_ik beta_k,  dF/dc_ik = -(1/eps) x_ik (G_ik - alpha_i - beta_k),
// with G_ik = r(u,i) e_k / Imp_i, applies Adam (ascent) to the tile and writes C and the moments
// back, then solves Sinkhorn on the new costs without reloading them from HBM. The Gram block is
// accumulated in registers for tiles of up to 21 columns (in passes of at most 64 entries) and from
// a shared copy of the policy otherwise; the (m-1) x (m-1) system is solved by one warp,
// lane-parallel in single precision for tiles of up to 21 columns (double-precision division and
// square root are long software sequences on this part) and in double precision for wider ones.
#pragma once
#include "fr_device.cuh"
#include "fr_internal.h"

namespace fr {

namespace {

struct Smem {
    float* gp;    // [ncx] g^(L-1)' of the previous solve (update modes)
    float* ib;    // [ncx] 1 / b_k
    float* e;     // [ncx] exposure
    float* beta;  // [ncx]
    float* coef;  // [2] Adam step size and sqrt of the second bias correction
    unsigned long long* bar;  // mbarrier of the staged copies
    float* red;   // reduction scratch (sweep double buffer / update reductions)
    float* out;   // [3*ncp + NG] reduction results
    double* A;    // [n*n] Gram system (update modes; floats for narrow tiles)
    double* rhs;  // [ncp]
    float* Lt;    // [n*n] transposed Cholesky factor (update modes, narrow tiles)
    float* C;     // [nc][ld] staged cost tile of the consumer
    float* r;     // [ld] staged relevance row
    float* om;    // [ld] dF/dImp_i (update modes)
    float* lse;   // [ld] row log2-normalisers of the previous policy (update modes)
    float* h;     // [ld]
    float* alpha; // [ld]
    float* X;     // [nc][ld] policy of the consumer (update modes, wide tiles only)
};

// The Gram block of diag(cs) - X^T X is accumulated in registers for tiles of up to 21 columns, in
// passes of at most 64 entries (re-forming the policy each pass); wider tiles keep a shared copy of
// the policy instead.
__host__ __device__ constexpr bool reg_gram(int ncb) { return ncb <= 21; }
__host__ __device__ constexpr int n_gram(int ncb) { return reg_gram(ncb) ? ncb * (ncb - 1) / 2 : 1; }
__host__ __device__ constexpr int gram_chunk(int ncb) {
    return (n_gram(ncb) + (n_gram(ncb) + 63) / 64 - 1) / ((n_gram(ncb) + 63) / 64);
}

__host__ __device__ inline int ncp_of(int nc) { return (nc + 3) / 4 * 4; }
// per-column shared arrays hold max(nc, NCB) entries (zero beyond nc) so that unrolled loops over
// the compiled column bucket read zeros, never a neighbouring array
__host__ __device__ inline int ncx_of(int nc, int ncb) { return ncp_of(nc > ncb ? nc : ncb); }

// ts (tile sweep, ts = the shared tile's column stride in floats, a compile-time constant >= ld;
// 0 for the register sweep, whose tile has stride ld): the Sinkhorn phase reads its costs from the
// staged tile, so the tile stays resident through the solve and the next consumer is staged after
// it; omega and the relevance row are then read from global memory (L2) and alpha overwrites h,
// which keeps a 1000-item CTA near 56 KB (four CTAs per SM).
__host__ __device__ inline size_t smem_layout(int ncb, int nc, int ld, int W, int mode, int ts,
                                              Smem* s, unsigned char* base) {
    const int P = pow2ceil(ncb);
    const int NG = n_gram(ncb);
    const int PG = pow2ceil(gram_chunk(ncb));
    const int ncp = ncp_of(nc);
    const int ncx = ncx_of(nc, ncb);
    const int n = nc - 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 15) / 16 * 16;
        return o;
    };
    const bool upd = mode != MODE_SWEEP;
    size_t red_f = (size_t)W * 3 * P;
    if ((size_t)W * PG > red_f) red_f = (size_t)W * PG;
    const size_t o_gp = take(sizeof(float) * ncx), o_ib = take(sizeof(float) * ncx);
    const size_t o_e = take(sizeof(float) * ncx), o_beta = take(sizeof(float) * ncx);
    const size_t o_coef = take(sizeof(float) * 2), o_bar = take(sizeof(unsigned long long));
    const size_t o_red = take(sizeof(float) * red_f);
    const size_t o_out = take(sizeof(float) * (3 * ncp + NG));
    const size_t o_C = take(sizeof(float) * (size_t)nc * (ts ? ts : ld));
    const size_t o_r = ts ? 0 : take(sizeof(float) * ld);
    size_t o_A = 0, o_rhs = 0, o_Lt = 0, o_om = 0, o_lse = 0, o_h = 0, o_al = 0, o_X = 0;
    if (upd) {
        o_A = take(sizeof(double) * (size_t)(n > 0 ? n * n : 1));
        o_rhs = take(sizeof(double) * ncp);
        o_Lt = take(sizeof(float) * (size_t)(n > 0 ? n * n : 1));
        o_om = ts ? 0 : take(sizeof(float) * ld);
        o_lse = take(sizeof(float) * ld);
        o_h = take(sizeof(float) * ld);
        o_al = ts ? o_h : take(sizeof(float) * ld);
        if (!reg_gram(ncb)) o_X = take(sizeof(float) * (size_t)nc * ld);
    }
    if (s) {
        s->gp = (float*)(base + o_gp);
        s->ib = (float*)(base + o_ib);
        s->e = (float*)(base + o_e);
        s->beta = (float*)(base + o_beta);
        s->coef = (float*)(base + o_coef);
        s->bar = (unsigned long long*)(base + o_bar);
        s->red = (float*)(base + o_red);
        s->out = (float*)(base + o_out);
        s->A = (double*)(base + o_A);
        s->rhs = (double*)(base + o_rhs);
        s->Lt = (float*)(base + o_Lt);
        s->C = (float*)(base + o_C);
        s->r = ts ? nullptr : (float*)(base + o_r);
        s->om = ts ? nullptr : (float*)(base + o_om);
        s->lse = (float*)(base + o_lse);
        s->h = (float*)(base + o_h);
        s->alpha = (float*)(base + o_al);
        s->X = (float*)(base + o_X);
    }
    return off;
}

// Thread 0: bulk-copies consumer un's cost tile (and, unless ts, its relevance row) into the
// staging buffers; with ts the tile's columns land ts floats apart (one copy per column). Every
// thread of the CTA must be done reading them (the caller sits after a __syncthreads).
__device__ __forceinline__ void stage_consumer(const P1Args& a, int un, int nc, int ld,
                                               const Smem& s, bool prefetch_moments, int ts) {
    if (un < 0 || un >= a.U) return;
    const unsigned tile = (unsigned)(sizeof(float) * (size_t)nc * ld);
    const unsigned row = (unsigned)(sizeof(float) * ld);
    fence_proxy_async_smem();
    if (ts) {
        // a column slot of the tile holds ts floats, at least the item count rounded up to 8; a
        // caller's row stride ld may be longer (the allocation-free entry point), and what lies
        // beyond the slot is padding, so each column copies min(ld, ts) floats (a multiple of 8)
        const int lc = ld < ts ? ld : ts;
        const unsigned rowc = (unsigned)(sizeof(float) * lc);
        mbar_arrive_expect_tx(s.bar, (unsigned)nc * rowc);
        for (int k = 0; k < nc; ++k)
            bulk_g2s(s.C + (size_t)k * ts, a.C + ((size_t)un * nc + k) * ld, rowc, s.bar);
    } else {
        mbar_arrive_expect_tx(s.bar, tile + row);
        bulk_g2s(s.C, a.C + (size_t)un * nc * ld, tile, s.bar);
        bulk_g2s(s.r, a.r + (size_t)un * ld, row, s.bar);
    }
    if (prefetch_moments) {  // the Adam moments of that consumer: into L2 for the gradient step
        bulk_prefetch_l2(a.m1 + (size_t)un * nc * ld, tile);
        bulk_prefetch_l2(a.m2 + (size_t)un * nc * ld, tile);
    }
}

// Thread 0, tile sweep: pulls consumer un's tile, relevance row and (update mode) Adam moments into
// L2 while the current consumer's solve still holds the shared tile.
__device__ __forceinline__ void prefetch_consumer(const P1Args& a, int un, int nc, int ld,
                                                  bool moments) {
    if (un < 0 || un >= a.U) return;
    const unsigned tile = (unsigned)(sizeof(float) * (size_t)nc * ld);
    bulk_prefetch_l2(a.C + (size_t)un * nc * ld, tile);
    bulk_prefetch_l2(a.r + (size_t)un * ld, (unsigned)(sizeof(float) * ld));
    if (moments) {
        bulk_prefetch_l2(a.m1 + (size_t)un * nc * ld, tile);
        bulk_prefetch_l2(a.m2 + (size_t)un * nc * ld, tile);
    }
}

// Gram entries Q0 .. Q0 + NQ - 1 (the upper triangle of the leading (NCB-1) x (NCB-1) block, row by
// row) of diag(cs) - X^T X over the consumer's rows, from the policy re-formed as
// x_ik = 2^(g'_k - c'_ik - lse_i); rows of x sum to 1, so the diagonal is sum_i x_ik (1 - x_ik)
// without cancellation. The CTA sums land in gout[Q0 ..]. Every thread of the CTA must call it.
template <int NCB, bool EXACT, int Q0, int NQ>
__device__ __forceinline__ void gram_pass(const Smem& s, int nc, int I, int lds, float sc,
                                          float* gout) {
    const int n = nc - 1;
    float gram[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) gram[q] = 0.f;
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        float x[NCB];
        const float l = s.lse[i];
#pragma unroll
        for (int k = 0; k < NCB; ++k)
            x[k] = (EXACT || k < nc) ? ex2(s.gp[k] - s.C[k * lds + i] * sc - l) : 0.f;
        int q = 0;
#pragma unroll
        for (int k = 0; k < NCB - 1; ++k) {
#pragma unroll
            for (int m = k; m < NCB - 1; ++m, ++q) {
                if (q >= Q0 && q < Q0 + NQ && (EXACT || m < n))
                    gram[q - Q0] += k == m ? x[k] * (1.f - x[k]) : -x[k] * x[m];
            }
        }
    }
    cta_reduce_vec<NQ>(gram, NQ, s.red, gout + Q0);
}

template <int NCB, bool EXACT, int Q0 = 0>
__device__ __forceinline__ void gram_block(const Smem& s, int nc, int I, int lds, float sc,
                                           float* gout) {
    constexpr int NGALL = n_gram(NCB), CH = gram_chunk(NCB);
    constexpr int NQ = NGALL - Q0 < CH ? NGALL - Q0 : CH;
    gram_pass<NCB, EXACT, Q0, NQ>(s, nc, I, lds, sc, gout);
    if constexpr (Q0 + NQ < NGALL) gram_block<NCB, EXACT, Q0 + NQ>(s, nc, I, lds, sc, gout);
}

// Whether a Sinkhorn iteration is the last one: BoolTag<B> decides at compile time (the peeled
// last iteration is its own instantiation), a plain bool at run time. BoolTag also selects the
// tile sweep's form.
template <bool B>
struct BoolTag {
    static constexpr bool value = B;
};
template <bool B>
__device__ __forceinline__ constexpr bool last_of(BoolTag<B>) { return B; }
__device__ __forceinline__ bool last_of(bool b) { return b; }

template <int BR>
struct RowBlock {  // one load / store of a block's BR consecutive floats (8- or 16-byte aligned)
    static __device__ __forceinline__ void load(const float* p, f2 (&c)[BR / 2]) {
        if constexpr (BR == 2) {
            const float2 v = *reinterpret_cast<const float2*>(p);
            c[0] = pk(v.x, v.y);
        } else {
            const float4 v = *reinterpret_cast<const float4*>(p);
            c[0] = pk(v.x, v.y);
            c[1] = pk(v.z, v.w);
        }
    }
    static __device__ __forceinline__ void store(float* p, const float (&v)[BR]) {
        if constexpr (BR == 2)
            *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
        else
            *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};

// Largest drift |g'_k - g0_k| (log2 units) of a column potential from its value at the start of
// the solve for which the sweeps keep their exponential form (the tile sweep below, and the
// register sweep of at most 11 columns in p1_kernel).
constexpr float TS_DRIFT = 30.f;

// Tile sweep: the Sinkhorn phase of consumer u with its costs read from the resident shared tile
// (the same iteration as the register sweep of p1_kernel). A thread owns R / BR blocks of BR
// consecutive rows (BR = 2 or 4), block b at rows BR (b T + tid): the read of a block's column k
// is one 8- or 16-byte load per lane and conflict-free (consecutive lanes, consecutive words), at
// a compile-time offset k LDS from the block's base (no address arithmetic per load), and no
// costs stay in registers between iterations, which is what allows eight rows per thread at four
// CTAs per SM. The impacts of a block's rows go straight into the partial row part_row (written by
// its first consumer, first_row, and accumulated by the later ones). (na, nu) is the consumer the
// CTA solves next (nu < 0: none), prefetched into L2 near the end of this solve.
//
// The tile holds one of two forms of the row-shifted kernel; both give the same policy in exact
// arithmetic (a factor per column or per row cancels in x_ik = p_ik / sum_k p_ik).
// - Exponential form (from the start of every solve): E_ik = 2^(g0_k - c~_ik) with g0 = g' at the
//   start, c~_ik = c_ik / (eps ln 2) + shift_i and shift_i = max_k (g0_k - c_ik / (eps ln 2)), so
//   the row's largest E is exactly 1 (padding rows I <= i < ld hold 0). An iteration forms
//   G_k = 2^(g'_k - g0_k), one ex2 per column, and p_ik = E_ik G_k, one multiply per cell. While
//   every |g'_k - g0_k| <= TS_DRIFT, a real row's sum lies in [2^-30, m 2^30], and a term flushed
//   to zero when E was formed (below 2^-126 of its row's largest) stays below 2^-66 of the row's
//   largest term: the result is the log form's up to FP32 rounding.
// - Log form: c~_ik in the tile (+inf on padding rows), p_ik = 2^(g'_k - c~_ik), one ex2 per cell,
//   rows re-shifted exactly when their sum leaves [2^-64, 2^64]. When a potential drifts past
//   TS_DRIFT the CTA rebuilds its rows in this form from the costs in global memory (at the
//   current g') and finishes the solve in it; every warp holds the same g', so all decide alike.
// Each thread rewrites only its own rows, which only it reads during the solve.
template <int NCB, int R, int BR, int LDS, bool EXACT, int MODE, bool REC = false>
__device__ __forceinline__ void tile_sweep(const P1Args& a, const Smem& s, int u, int nc,
                                           float (&gm)[(NCB + 31) / 32], int& par,
                                           float* part_row, bool first_row, const P1Args& na,
                                           int nu) {
    static_assert((BR == 2 || BR == 4) && R % BR == 0, "blocks of two or four rows");
    constexpr int GPL = (NCB + 31) / 32;
    constexpr int NB = R / BR, NP = BR / 2;
    using RBk = RowBlock<BR>;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int T = blockDim.x, I = a.I, ld = a.ld;
    const float sc = a.inv_eps_ln2;
    // Block b starts at row rb = BR (b T + tid); ld is a multiple of 8, so a block lies inside the
    // tile (rb < ld) or past it. Row j of the block is a consumer row if rb + j < I.
    //
    // Rows rb .. rb + BR - 1: reads their costs at cb + k cstride (column k; the shared tile, or the
    // consumer's costs in global memory), shifts each row at potentials gk and writes to the tile
    // at cd + k LDS either E (form BoolTag<true>) or c~ (BoolTag<false>).
    auto shift_rows = [&](const float* cb, int cstride, float* cd, int rb, const float (&gk)[NCB],
                          auto form) {
        constexpr bool EXPF = decltype(form)::value;
        float M[BR];
#pragma unroll
        for (int j = 0; j < BR; ++j) M[j] = -INFINITY;
#pragma unroll
        for (int k = 0; k < NCB; ++k) {
            if (EXACT || k < nc) {
                f2 c[NP];
                RBk::load(cb + k * cstride, c);
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    float c0, c1;
                    upk(c[q], c0, c1);
                    M[2 * q] = fmaxf(M[2 * q], gk[k] - c0 * sc);
                    M[2 * q + 1] = fmaxf(M[2 * q + 1], gk[k] - c1 * sc);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NCB; ++k) {
            if (EXACT || k < nc) {
                f2 c[NP];
                RBk::load(cb + k * cstride, c);
                float v[BR];
#pragma unroll
                for (int q = 0; q < NP; ++q) upk(c[q], v[2 * q], v[2 * q + 1]);
#pragma unroll
                for (int j = 0; j < BR; ++j) {
                    if constexpr (EXPF)
                        v[j] = rb + j < I ? ex2(gk[k] - fmaf(v[j], sc, M[j])) : 0.f;
                    else
                        v[j] = rb + j < I ? fmaf(v[j], sc, M[j]) : INFINITY;
                }
                RBk::store(cd + k * LDS, v);
            }
        }
    };
    float g0m[GPL];  // g' at the start of the solve (this lane's columns)
#pragma unroll
    for (int j = 0; j < GPL; ++j) g0m[j] = gm[j];
    {
        float gk[NCB];
        bcast_g<NCB, GPL>(gm, gk);
#pragma unroll 1
        for (int b = 0; b < NB; ++b) {
            const int rb = BR * (b * T + tid);
            if (rb >= ld) break;
            shift_rows(s.C + rb, LDS, s.C + rb, rb, gk, BoolTag<true>{});
        }
    }
    bool lg = false;  // the tile holds the log form (the same in every thread of the CTA)
    const float* __restrict__ Cu = a.C + (size_t)u * nc * ld;
    // One iteration; the last one (which also writes g^(L-1) and adds the impacts) is a separate
    // instantiation, so the loop over the first L - 1 carries no test for it.
    auto iteration = [&](int l, auto tag) {
        constexpr bool last = decltype(tag)::value;
        if (last && warp == 0) {
#pragma unroll
            for (int j = 0; j < GPL; ++j)
                if (j * 32 + lane < nc) a.gP[(size_t)u * nc + j * 32 + lane] = gm[j];
        }
        if (!lg) {
            bool far = false;
#pragma unroll
            for (int j = 0; j < GPL; ++j)
                if (j * 32 + lane < nc) far |= !(fabsf(gm[j] - g0m[j]) <= TS_DRIFT);
            if (__builtin_expect(__any_sync(FULL, far), 0)) {  // rebuild the rows in the log form
                lg = true;
                if (tid == 0) atomicAdd(&a.st->log_solves, 1ull);
                float gk[NCB];
                bcast_g<NCB, GPL>(gm, gk);
#pragma unroll 1
                for (int b = 0; b < NB; ++b) {
                    const int rb = BR * (b * T + tid);
                    if (rb >= ld) break;
                    shift_rows(Cu + rb, ld, s.C + rb, rb, gk, BoolTag<false>{});
                }
            }
        }
        // Tiles of up to 16 columns hold g' (or G) as packed pairs and the column sums as packed
        // row-pair partials; wider tiles hold both as scalars (pairs formed at use, column sums
        // accumulated with two FMAs), which keeps 21 columns within the register budget.
        constexpr bool WIDE = NCB > 16;
        f2 cs2[WIDE ? 1 : NCB];
        float csw[WIDE ? NCB : 1];
#pragma unroll
        for (int k = 0; k < (WIDE ? 1 : NCB); ++k) cs2[k] = 0ull;
#pragma unroll
        for (int k = 0; k < (WIDE ? NCB : 1); ++k) csw[k] = 0.f;
        auto sweep = [&](auto form) {
            constexpr bool EXPF = decltype(form)::value;
            // two blocks in flight for wide tiles (21 columns: 4 % faster), one for 11 columns
            // (two were 1-3 % slower there)
            constexpr int UB = WIDE ? 2 : 1;
            float gk[NCB];  // G_k (exponential form) or g'_k (log form)
            if constexpr (EXPF) {
                float Gm[GPL];
#pragma unroll
                for (int j = 0; j < GPL; ++j) Gm[j] = ex2(gm[j] - g0m[j]);
                bcast_g<NCB, GPL>(Gm, gk);
            } else {
                bcast_g<NCB, GPL>(gm, gk);
            }
            f2 g2[WIDE ? 1 : NCB];
            if constexpr (!WIDE) {
#pragma unroll
                for (int k = 0; k < NCB; ++k) g2[k] = pk(gk[k], gk[k]);
            } else {
                (void)g2;
            }
            auto gpair = [&](int k) -> f2 {
                if constexpr (WIDE) return pk(gk[k], gk[k]);
                else return g2[k];
            };
            auto gscal = [&](int k) -> float {
                if constexpr (WIDE) {
                    return gk[k];
                } else {
                    float lo, hi;
                    upk(g2[k], lo, hi);
                    return lo;
                }
            };
#pragma unroll UB
            for (int b = 0; b < NB; ++b) {
                const int rb = BR * (b * T + tid);
                if (rb >= ld) break;
                float* cb = s.C + rb;
                f2 p[NP][NCB];  // row pairs (0, 1) and (2, 3) of the block
                f2 S2[NP];
#pragma unroll
                for (int q = 0; q < NP; ++q) S2[q] = 0ull;
#pragma unroll
                for (int k = 0; k < NCB; ++k) {
                    if (EXACT || k < nc) {
                        f2 c[NP];
                        RBk::load(cb + k * LDS, c);
#pragma unroll
                        for (int q = 0; q < NP; ++q) {
                            if constexpr (EXPF) {
                                p[q][k] = mul2(c[q], gpair(k));
                            } else {
                                float d0, d1;
                                upk(sub2(gpair(k), c[q]), d0, d1);
                                p[q][k] = pk(ex2(d0), ex2(d1));
                            }
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < NP; ++q) p[q][k] = 0ull;
                    }
#pragma unroll
                    for (int q = 0; q < NP; ++q) S2[q] = add2(S2[q], p[q][k]);
                }
                float S[BR];
#pragma unroll
                for (int q = 0; q < NP; ++q) upk(S2[q], S[2 * q], S[2 * q + 1]);
                if constexpr (!EXPF) {
                    bool bad[BR], any_bad = false;
#pragma unroll
                    for (int j = 0; j < BR; ++j) {
                        bad[j] = rb + j < I && !(S[j] >= 0x1p-64f && S[j] <= 0x1p64f);
                        any_bad |= bad[j];
                    }
                    if (__builtin_expect(any_bad, 0)) {  // re-shift the block's out-of-range rows
                        float M[BR];
#pragma unroll
                        for (int j = 0; j < BR; ++j) M[j] = -INFINITY;
#pragma unroll
                        for (int k = 0; k < NCB; ++k) {
                            if (EXACT || k < nc) {
                                const float gkk = gscal(k);
                                f2 c[NP];
                                RBk::load(cb + k * LDS, c);
#pragma unroll
                                for (int q = 0; q < NP; ++q) {
                                    float c0, c1;
                                    upk(c[q], c0, c1);
                                    M[2 * q] = fmaxf(M[2 * q], gkk - c0);
                                    M[2 * q + 1] = fmaxf(M[2 * q + 1], gkk - c1);
                                }
                            }
                        }
#pragma unroll
                        for (int j = 0; j < BR; ++j) M[j] = bad[j] ? M[j] : 0.f;
#pragma unroll
                        for (int q = 0; q < NP; ++q) S2[q] = 0ull;
#pragma unroll
                        for (int k = 0; k < NCB; ++k) {
                            if (EXACT || k < nc) {
                                f2 c[NP];
                                RBk::load(cb + k * LDS, c);
                                float v[BR];
#pragma unroll
                                for (int q = 0; q < NP; ++q) {
                                    upk(c[q], v[2 * q], v[2 * q + 1]);
                                    v[2 * q] += M[2 * q];
                                    v[2 * q + 1] += M[2 * q + 1];
                                    float d0, d1;
                                    upk(sub2(gpair(k), pk(v[2 * q], v[2 * q + 1])), d0, d1);
                                    p[q][k] = pk(ex2(d0), ex2(d1));
                                }
                                RBk::store(cb + k * LDS, v);
                            }
#pragma unroll
                            for (int q = 0; q < NP; ++q) S2[q] = add2(S2[q], p[q][k]);
                        }
#pragma unroll
                        for (int q = 0; q < NP; ++q) upk(S2[q], S[2 * q], S[2 * q + 1]);
                    }
                }
                float inv[BR];
#pragma unroll
                for (int j = 0; j < BR; ++j) inv[j] = rb + j < I ? rcp_approx(S[j]) : 0.f;
#pragma unroll
                for (int q = 0; q < NP; ++q) {
                    const f2 i2 = pk(inv[2 * q], inv[2 * q + 1]);
#pragma unroll
                    for (int k = 0; k < NCB; ++k) {
                        if constexpr (WIDE) {
                            float p0, p1;
                            upk(p[q][k], p0, p1);
                            csw[k] = fmaf(p1, inv[2 * q + 1], fmaf(p0, inv[2 * q], csw[k]));
                        } else {
                            cs2[k] = fma2(p[q][k], i2, cs2[k]);
                        }
                    }
                }
                if (last) {  // impacts: r(u,i) sum_{k<K} e_k x_ik for the block's rows
                    float w[BR];
#pragma unroll
                    for (int j = 0; j < BR; ++j) w[j] = 0.f;
#pragma unroll
                    for (int k = 0; k < NCB; ++k) {
                        if (k < a.K) {
                            const float ek = s.e[k];
#pragma unroll
                            for (int q = 0; q < NP; ++q) {
                                float p0, p1;
                                upk(p[q][k], p0, p1);
                                w[2 * q] += ek * p0;
                                w[2 * q + 1] += ek * p1;
                            }
                        }
                    }
                    float* pp = part_row + rb;
                    f2 rr[NP], acc[NP];
                    RBk::load(a.r + (size_t)u * ld + rb, rr);
                    if (first_row) {
#pragma unroll
                        for (int q = 0; q < NP; ++q) acc[q] = 0ull;
                    } else {
                        RBk::load(pp, acc);
                    }
                    float v[BR];
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        float r0, r1, a0, a1;
                        upk(rr[q], r0, r1);
                        upk(acc[q], a0, a1);
                        v[2 * q] = a0 + r0 * (w[2 * q] * inv[2 * q]);
                        v[2 * q + 1] = a1 + r1 * (w[2 * q + 1] * inv[2 * q + 1]);
                    }
                    RBk::store(pp, v);
                }
            }
        };
        if (__builtin_expect(lg, 0))
            sweep(BoolTag<false>{});
        else
            sweep(BoolTag<true>{});
        float cs[NCB];
#pragma unroll
        for (int k = 0; k < NCB; ++k) {
            if constexpr (WIDE) {
                cs[k] = csw[k];
            } else {
                float lo, hi;
                upk(cs2[k], lo, hi);
                cs[k] = lo + hi;
            }
        }
        column_update<NCB, GPL, REC>(cs, gm, nc, s.red, s.ib, par, lane, warp, W,
                                     REC ? a.gall + ((size_t)u * a.L + l) * nc : nullptr,
                                     REC ? a.csall + ((size_t)u * a.L + l) * nc : nullptr);
        par ^= 1;
        // the next consumer's tile and relevance row into L2 eight iterations before the end of
        // this solve: early enough to hide the HBM latency, late enough that four CTAs per SM
        // prefetching at once do not evict them again before the copy after the solve (its Adam
        // moments follow at the start of its gradient step, closer to their use)
        if (l == (a.L > 8 ? a.L - 8 : 0) && tid == 0)
            prefetch_consumer(na, nu, EXACT ? NCB : na.nc, na.ld, false);
    };
    for (int l = 0; l < a.L - 1; ++l) iteration(l, BoolTag<false>{});
    iteration(a.L - 1, BoolTag<true>{});
}

// One consumer u of market a, as one step of a CTA's persistent loop: the gradient step (update
// modes) and the Sinkhorn solve (sweep modes). The consumer's tile was staged into shared memory
// by the previous step (or before the loop); (na, nu) is the consumer this CTA solves next (nu < 0:
// none), whose tile this step stages. Impacts go into part_row (the tile sweep: written by the
// row's first consumer, first_row) or are added to acc_imp (the register sweep; the caller writes
// them out); the squared gradient is added to gn2. Returns false if a bounded wait expired (the CTA
// then stops). The per-market shared arrays (e, 1/b, omega, the Adam coefficients) must hold a's.
template <int NCB, int R, bool EXACT, int MODE, int TS, bool REC = false>
__device__ __forceinline__ bool p1_consumer(const P1Args& a, const Smem& s, int u, const P1Args& na,
                                            int nu, float* part_row, bool first_row,
                                            float (&acc_imp)[R], double& gn2, int& par,
                                            unsigned& phase) {
    constexpr int GPL = (NCB + 31) / 32;
    constexpr bool REG_GRAM = reg_gram(NCB);
    constexpr bool PAIR = R % 2 == 0;
    const int nc = EXACT ? NCB : a.nc;
    const int ncn = EXACT ? NCB : na.nc;
    const int ncp = ncp_of(nc);
    const int ncx = ncx_of(nc, NCB);
    const int n = nc - 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int T = blockDim.x;
    const int I = a.I, ld = a.ld;
    const int i0 = tid * R;
    const bool any_row = i0 < I;
    const float sc = a.inv_eps_ln2;
    const int lds = TS ? TS : ld;  // column stride of the shared tile
    (void)ncn;
    (void)n;
    (void)any_row;
    (void)ncx;
    // omega_i: the staged copy, or (tile sweep) global memory; omega has ld entries, zero beyond I
    auto om_at = [&](int i) { return TS ? __ldg(a.omega + i) : s.om[i]; };
    {
            const size_t tile = (size_t)u * nc * ld;
            const float* __restrict__ r_u = a.r + (size_t)u * ld;
            auto r_at = [&](int i) { return TS ? __ldg(r_u + i) : s.r[i]; };
            float gm[GPL];  // column potentials of the columns this lane holds (same in every warp)
    #pragma unroll
            for (int j = 0; j < GPL; ++j) {
                const int col = j * 32 + lane;
                gm[j] = (a.warm && col < nc) ? a.gL[(size_t)u * nc + col] : 0.f;
                // the potentials this solve starts from, for the unrolled gradient's forward re-run
                if (MODE != MODE_GRAD && a.g0 && warp == 0 && col < nc) a.g0[(size_t)u * nc + col] = gm[j];
            }
            if (MODE != MODE_SWEEP && tid < ncx) s.gp[tid] = tid < nc ? a.gP[(size_t)u * nc + tid] : 0.f;
            // the consumer's tile was staged one consumer ago (the register sweep) or right after the
            // previous solve (the tile sweep), and it is the only copy in flight. The wait is bounded:
            // if it expires, the CTA records a timeout, waits (with the default bound) for the copy to
            // land and stops, so that no bulk copy is still writing into its shared memory when it
            // leaves. In the tile sweep's update modes the first gradient pass reads the costs from
            // global memory (L2, where the previous solve prefetched them) while the copy lands, and
            // the wait follows that pass.
            constexpr bool LATE_WAIT = TS != 0 && MODE != MODE_SWEEP;
            bool tile_ok = true;  // the same in every thread (cta_wait_or_drain)
            if constexpr (!LATE_WAIT) {
                tile_ok = cta_wait_or_drain(s.bar, phase, a.max_polls, kDefaultPolls, &a.st->err, 4);
                phase ^= 1u;
            } else {
                __syncthreads();  // s.gp / s.e / s.ib / s.om / s.coef visible
            }
            if (!tile_ok) return false;

            if constexpr (MODE != MODE_SWEEP) {
                if (TS && MODE == MODE_UPDATE_SWEEP && a.optimizer == 0 && tid == 0) {
                    // the consumer's Adam moments into L2 while the gradient passes run
                    const unsigned tb = (unsigned)(sizeof(float) * (size_t)nc * ld);
                    bulk_prefetch_l2(a.m1 + tile, tb);
                    bulk_prefetch_l2(a.m2 + tile, tb);
                }
                // ---------------- gradient of F at the previous policy ------------------------------
                // x_ik = 2^(g'_k - c'_ik - lse_i) is re-formed from the staged tile and the row
                // log-normaliser lse_i of the first pass.
                {
                    float acc[3][NCB];  // q, cs, X^T h partials
    #pragma unroll
                    for (int k = 0; k < NCB; ++k) acc[0][k] = acc[1][k] = acc[2][k] = 0.f;
                    for (int i = tid; i < I; i += T) {
                        float x[NCB];
                        float M = -INFINITY;
    #pragma unroll
                        for (int k = 0; k < NCB; ++k) {
                            float c = 0.f;
                            if (EXACT || k < nc)
                                c = LATE_WAIT ? __ldcg(a.C + tile + (size_t)k * ld + i) : s.C[k * lds + i];
                            x[k] = (EXACT || k < nc) ? s.gp[k] - c * sc : -INFINITY;
                            M = fmaxf(M, x[k]);
                        }
                        float S = 0.f;
    #pragma unroll
                        for (int k = 0; k < NCB; ++k) {
                            x[k] = ex2(x[k] - M);
                            S += x[k];
                        }
                        const float inv = rcp_approx(S);  // S in [1, m]: the row max contributes 1
                        const float wr = om_at(i) * r_at(i);  // dF/dx_ik = wr_i e_k
                        float hh = 0.f, vi = 0.f;
    #pragma unroll
                        for (int k = 0; k < NCB; ++k) {
                            x[k] *= inv;
                            hh += x[k] * (wr * s.e[k]);
                            if (MODE == MODE_GRAD && k < a.K) vi += s.e[k] * x[k];
                        }
    #pragma unroll
                        for (int k = 0; k < NCB; ++k) {
                            acc[0][k] += x[k] * (wr * s.e[k]);
                            acc[1][k] += x[k];
                            acc[2][k] += x[k] * hh;
                            if constexpr (!REG_GRAM) {
                                if (EXACT || k < nc) s.X[k * ld + i] = x[k];
                            }
                        }
                        s.lse[i] = M + lg2_approx(S);
                        s.h[i] = hh;
                        // dF/dr(u,i) = (dF/dImp_i) sum_{k<K} e_k x_ik (C does not depend on r)
                        if (MODE == MODE_GRAD && a.dr) a.dr[(size_t)u * I + i] = om_at(i) * vi;
                    }
                    cta_reduce<NCB, 3>(acc, nc, s.red, s.out, ncp);  // s.out: [q | cs | X^T h]
                }
                if constexpr (LATE_WAIT) {  // the shared tile from here on
                    tile_ok = cta_wait_or_drain(s.bar, phase, a.max_polls, kDefaultPolls, &a.st->err, 4);
                    phase ^= 1u;
                    if (!tile_ok) return false;
                }
                // Gram block M[0:n,0:n] of diag(cs) - X^T X; rows of x sum to 1, so the diagonal is
                // sum_i x_ik (1 - x_ik) without cancellation.
                if constexpr (REG_GRAM) {
                    float* gout = s.out + 3 * ncp;
                    gram_block<NCB, EXACT>(s, nc, I, lds, sc, gout);
                    float* Af = reinterpret_cast<float*>(s.A);
                    float* rf = reinterpret_cast<float*>(s.rhs);
                    for (int idx = tid; idx < n * n; idx += T) {
                        int k = idx / n, m = idx % n;
                        if (k > m) { const int t = k; k = m; m = t; }
                        Af[idx] = gout[k * (NCB - 1) - k * (k - 1) / 2 + (m - k)];
                    }
                    for (int k = tid; k < ncx; k += T) {
                        if (k < n) rf[k] = s.out[k] - s.out[2 * ncp + k];
                        s.beta[k] = 0.f;
                    }
                    __syncthreads();
                    if (warp == 0) warp_cholesky_solve_f32<NCB - 1>(Af, rf, n, s.Lt, s.beta, lane);
                    __syncthreads();
                } else {
                    for (int pidx = warp; pidx < n * (n + 1) / 2; pidx += W) {
                        int k = 0, rem = pidx;
                        while (rem >= n - k) { rem -= n - k; ++k; }
                        const int m = k + rem;
                        const float* xk = s.X + k * ld;
                        const float* xm = s.X + m * ld;
                        float sum = 0.f;
                        if (k == m) {
                            for (int i = lane; i < I; i += 32) sum += xk[i] * (1.f - xk[i]);
                        } else {
                            for (int i = lane; i < I; i += 32) sum -= xk[i] * xm[i];
                        }
    #pragma unroll
                        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
                        if (lane == 0) {
                            s.A[k * n + m] = (double)sum;
                            s.A[m * n + k] = (double)sum;
                        }
                    }
                    for (int k = tid; k < n; k += T)
                        s.rhs[k] = (double)s.out[k] - (double)s.out[2 * ncp + k];
                    __syncthreads();
                    if (warp == 0) warp_cholesky_solve(s.A, s.rhs, n, lane);
                    __syncthreads();
                    for (int k = tid; k < ncx; k += T) s.beta[k] = k < n ? (float)s.rhs[k] : 0.f;
                    __syncthreads();
                }
                // alpha_i = h_i - sum_k x_ik beta_k
                for (int i = tid; i < I; i += T) {
                    const float l = s.lse[i];
                    float sb = 0.f;
    #pragma unroll
                    for (int k = 0; k < NCB; ++k)
                        if (EXACT || k < nc) sb += ex2(s.gp[k] - s.C[k * lds + i] * sc - l) * s.beta[k];
                    s.alpha[i] = s.h[i] - sb;
                }
                __syncthreads();
                // gradient and Adam over the tile: each thread takes four consecutive items (float4)
                // and runs through the columns, so the per-item values (lse, alpha, omega r) are read
                // once per four items and eleven columns, and no index needs a division
                const float step_size = s.coef[0], inv_bc2s = 1.f / s.coef[1];
                float* __restrict__ Cg = a.C;
                float* __restrict__ m1g = a.m1;
                float* __restrict__ m2g = a.m2;
                float gsq = 0.f;
                for (int i4 = tid; i4 * 4 < I; i4 += T) {
                    const int i = i4 * 4;
                    const float4 l4 = reinterpret_cast<const float4*>(s.lse)[i4];
                    const float4 a4 = reinterpret_cast<const float4*>(s.alpha)[i4];
                    const float4 o4 = TS ? __ldg(reinterpret_cast<const float4*>(a.omega) + i4)
                                         : reinterpret_cast<const float4*>(s.om)[i4];
                    const float4 r4 = TS ? __ldg(reinterpret_cast<const float4*>(r_u) + i4)
                                         : reinterpret_cast<const float4*>(s.r)[i4];
                    const float lv[4] = {l4.x, l4.y, l4.z, l4.w}, av[4] = {a4.x, a4.y, a4.z, a4.w};
                    const float wv[4] = {o4.x * r4.x, o4.y * r4.y, o4.z * r4.z, o4.w * r4.w};
                    // Adam moments two columns ahead (their loads would otherwise wait for the stores
                    // of the previous column: the compiler cannot tell the addresses apart)
                    constexpr bool ADAM = MODE == MODE_UPDATE_SWEEP;
                    const bool adam = ADAM && a.optimizer == 0;
                    const int ncc = EXACT ? NCB : nc;
                    float4 mA = make_float4(0.f, 0.f, 0.f, 0.f), vA = mA, mB = mA, vB = mA;
                    auto ldmv = [&](int k, float4& m, float4& v) {
                        const size_t off = tile + (size_t)k * ld + i;
                        m = *reinterpret_cast<const float4*>(m1g + off);
                        v = *reinterpret_cast<const float4*>(m2g + off);
                    };
                    if (adam) {
                        ldmv(0, mA, vA);
                        if (1 < ncc) ldmv(1, mB, vB);
                    }
    #pragma unroll 4
                    for (int k = 0; k < NCB; ++k) {
                        if (!EXACT && k >= nc) break;
                        const float4 mm4 = mA, vv4 = vA;
                        mA = mB;
                        vA = vB;
                        if (adam && k + 2 < ncc) ldmv(k + 2, mB, vB);
                        const int qs = k * (lds / 4) + i4;  // float4 index in the shared tile
                        const float4 c4 = reinterpret_cast<const float4*>(s.C)[qs];
                        const float gpk = s.gp[k], ek = s.e[k], bk = s.beta[k];
                        float cv[4] = {c4.x, c4.y, c4.z, c4.w};
                        float gr[4];
    #pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const bool valid = i + j < I;
                            const float x = valid ? ex2(gpk - cv[j] * sc - lv[j]) : 0.f;
                            gr[j] = valid ? -a.inv_eps * x * (wv[j] * ek - av[j] - bk) : 0.f;
                            gsq += gr[j] * gr[j];
                        }
                        if constexpr (MODE == MODE_GRAD) {
    #pragma unroll
                            for (int j = 0; j < 4; ++j)
                                if (i + j < I) a.dC[((size_t)u * I + i + j) * nc + k] = gr[j];
                        } else {
                            const size_t off = tile + (size_t)k * ld + i;
                            if (a.optimizer == 1) {
    #pragma unroll
                                for (int j = 0; j < 4; ++j) cv[j] += a.lr * gr[j];
                            } else {
                                float mm[4] = {mm4.x, mm4.y, mm4.z, mm4.w};
                                float vv[4] = {vv4.x, vv4.y, vv4.z, vv4.w};
    #pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    mm[j] = a.beta1 * mm[j] + (1.f - a.beta1) * gr[j];
                                    vv[j] = a.beta2 * vv[j] + (1.f - a.beta2) * gr[j] * gr[j];
                                    // sqrt(v) / bc2s + eps with MUFU rsqrt / rcp (IEEE sqrt and
                                    // division are long instruction sequences on the per-cell path)
                                    const float sq = vv[j] > 0.f ? vv[j] * rsqrtf(vv[j]) : 0.f;
                                    cv[j] += __fdividef(step_size * mm[j], fmaf(sq, inv_bc2s, a.adam_eps));
                                }
                                *reinterpret_cast<float4*>(m1g + off) = make_float4(mm[0], mm[1], mm[2], mm[3]);
                                *reinterpret_cast<float4*>(m2g + off) = make_float4(vv[0], vv[1], vv[2], vv[3]);
                            }
                            const float4 cn = make_float4(cv[0], cv[1], cv[2], cv[3]);
                            *reinterpret_cast<float4*>(Cg + off) = cn;
                            reinterpret_cast<float4*>(s.C)[qs] = cn;
                        }
                    }
                }
                gn2 += (double)gsq;
                if constexpr (MODE == MODE_GRAD) {
                    __syncthreads();
                    if (tid == 0) stage_consumer(na, nu, ncn, na.ld, s, false, TS);
                    return true;  // no solve in gradient mode
                }
                __syncthreads();  // updated tile visible
            }

            // ---------------- Sinkhorn solve on the consumer's (new) costs ----------------------------
            if constexpr (TS != 0) {
                tile_sweep<NCB, R, 2, TS, EXACT, MODE, REC>(a, s, u, nc, gm, par, part_row, first_row, na, nu);
            } else {
            float rr[R];
            bool vr[R];
    #pragma unroll
            for (int r = 0; r < R; ++r) rr[r] = 0.f;
            if (any_row) ldv<R>(rr, s.r + i0);
    #pragma unroll
            for (int r = 0; r < R; ++r) vr[r] = i0 + r < I;
            float c[R][NCB];
            {
                float gk[NCB];
                bcast_g<NCB, GPL>(gm, gk);
    #pragma unroll
                for (int k = 0; k < NCB; ++k) {
                    float tmp[R];
    #pragma unroll
                    for (int r = 0; r < R; ++r) tmp[r] = 0.f;
                    if ((EXACT || k < nc) && any_row) ldv<R>(tmp, s.C + k * lds + i0);
    #pragma unroll
                    for (int r = 0; r < R; ++r) c[r][k] = tmp[r];
                }
    #pragma unroll
                for (int r = 0; r < R; ++r) {
                    float M = 0.f;
                    if (vr[r]) {
                        M = -INFINITY;
    #pragma unroll
                        for (int k = 0; k < NCB; ++k)
                            if (EXACT || k < nc) M = fmaxf(M, gk[k] - c[r][k] * sc);
                    }
    #pragma unroll
                    for (int k = 0; k < NCB; ++k)
                        c[r][k] = (vr[r] && (EXACT || k < nc)) ? c[r][k] * sc + M : INFINITY;
                }
            }
            // the last iteration (which also writes g^(L-1) and adds the impacts) as a separate
            // instantiation, where a second copy of the body fits the registers
            constexpr bool PEEL = NCB <= 11;
            if constexpr (PAIR) {
                constexpr int RP = R / 2;
                // Up to 11 columns the pairs start in the exponential form of the tile sweep (E pairs in
                // c2, G_k = 2^(g'_k - g0_k) per iteration, one packed multiply per two cells) and switch
                // to the log form (c~ pairs rebuilt from the costs in global memory at the current g')
                // when a potential drifts past TS_DRIFT; wider buckets keep the log form throughout.
                constexpr bool EXPF_OK = NCB <= 11;
                float g0m[GPL];  // g' at the start of the solve (this lane's columns)
    #pragma unroll
                for (int j = 0; j < GPL; ++j) g0m[j] = gm[j];
                f2 c2[RP][NCB];
                {
                    float gk[NCB];
                    bcast_g<NCB, GPL>(gm, gk);
    #pragma unroll
                    for (int rp = 0; rp < RP; ++rp)
    #pragma unroll
                        for (int k = 0; k < NCB; ++k) {
                            if constexpr (EXPF_OK)  // rows and columns outside the tile: c~ = inf, E = 0
                                c2[rp][k] = pk(ex2(gk[k] - c[2 * rp][k]), ex2(gk[k] - c[2 * rp + 1][k]));
                            else
                                c2[rp][k] = pk(c[2 * rp][k], c[2 * rp + 1][k]);
                        }
                }
                bool lg = !EXPF_OK;  // c2 holds the log form (the same in every thread of the CTA)
                auto iteration = [&](int l, auto tag) {
                    const bool last = last_of(tag);
                    if (last && warp == 0) {
    #pragma unroll
                        for (int j = 0; j < GPL; ++j)
                            if (j * 32 + lane < nc) a.gP[(size_t)u * nc + j * 32 + lane] = gm[j];
                    }
                    if constexpr (EXPF_OK) {
                        if (!lg) {
                            bool far = false;
    #pragma unroll
                            for (int j = 0; j < GPL; ++j)
                                if (j * 32 + lane < nc) far |= !(fabsf(gm[j] - g0m[j]) <= TS_DRIFT);
                            if (__builtin_expect(__any_sync(FULL, far), 0)) {  // rebuild in the log form
                                lg = true;
                                if (tid == 0) atomicAdd(&a.st->log_solves, 1ull);
                                float gk[NCB];
                                bcast_g<NCB, GPL>(gm, gk);
                                float cc[R][NCB];
    #pragma unroll
                                for (int k = 0; k < NCB; ++k) {
                                    float tmp[R];
    #pragma unroll
                                    for (int r = 0; r < R; ++r) tmp[r] = 0.f;
                                    if ((EXACT || k < nc) && any_row) ldv<R>(tmp, a.C + tile + (size_t)k * ld + i0);
    #pragma unroll
                                    for (int r = 0; r < R; ++r) cc[r][k] = tmp[r];
                                }
    #pragma unroll
                                for (int r = 0; r < R; ++r) {
                                    float M = 0.f;
                                    if (vr[r]) {
                                        M = -INFINITY;
    #pragma unroll
                                        for (int k = 0; k < NCB; ++k)
                                            if (EXACT || k < nc) M = fmaxf(M, gk[k] - cc[r][k] * sc);
                                    }
    #pragma unroll
                                    for (int k = 0; k < NCB; ++k)
                                        cc[r][k] = (vr[r] && (EXACT || k < nc)) ? cc[r][k] * sc + M : INFINITY;
                                }
    #pragma unroll
                                for (int rp = 0; rp < RP; ++rp)
    #pragma unroll
                                    for (int k = 0; k < NCB; ++k) c2[rp][k] = pk(cc[2 * rp][k], cc[2 * rp + 1][k]);
                            }
                        }
                    }
                    f2 cs2[NCB];
    #pragma unroll
                    for (int k = 0; k < NCB; ++k) cs2[k] = 0ull;
                    auto sweep = [&](auto form) {
                        constexpr bool EXPF = decltype(form)::value;
                        f2 g2[NCB];  // (G_k, G_k) in the exponential form, (g'_k, g'_k) in the log form
                        {
                            float gk[NCB];
                            if constexpr (EXPF) {
                                float Gm[GPL];
    #pragma unroll
                                for (int j = 0; j < GPL; ++j) Gm[j] = ex2(gm[j] - g0m[j]);
                                bcast_g<NCB, GPL>(Gm, gk);
                            } else {
                                bcast_g<NCB, GPL>(gm, gk);
                            }
    #pragma unroll
                            for (int k = 0; k < NCB; ++k) g2[k] = pk(gk[k], gk[k]);
                        }
    #pragma unroll
                        for (int rp = 0; rp < RP; ++rp) {
                            const bool v0 = vr[2 * rp], v1 = vr[2 * rp + 1];
                            f2 p2[NCB];
                            f2 S2 = 0ull;
    #pragma unroll
                            for (int k = 0; k < NCB; ++k) {
                                if constexpr (EXPF) {
                                    p2[k] = mul2(c2[rp][k], g2[k]);
                                } else {
                                    float d0, d1;
                                    upk(sub2(g2[k], c2[rp][k]), d0, d1);
                                    p2[k] = pk(ex2(d0), ex2(d1));
                                }
                                S2 = add2(S2, p2[k]);
                            }
                            float S0, S1;
                            upk(S2, S0, S1);
                            if constexpr (!EXPF) {
                                const bool bad0 = v0 && !(S0 >= 0x1p-64f && S0 <= 0x1p64f);
                                const bool bad1 = v1 && !(S1 >= 0x1p-64f && S1 <= 0x1p64f);
                                if (bad0 || bad1) {  // re-shift the pair's rows exactly
                                    float M0 = -INFINITY, M1 = -INFINITY;
    #pragma unroll
                                    for (int k = 0; k < NCB; ++k) {
                                        if (EXACT || k < nc) {
                                            float gkk, gdup, c0, c1;
                                            upk(g2[k], gkk, gdup);
                                            upk(c2[rp][k], c0, c1);
                                            M0 = fmaxf(M0, gkk - c0);
                                            M1 = fmaxf(M1, gkk - c1);
                                        }
                                    }
                                    const f2 M2 = pk(bad0 ? M0 : 0.f, bad1 ? M1 : 0.f);
                                    S2 = 0ull;
    #pragma unroll
                                    for (int k = 0; k < NCB; ++k) {
                                        if (EXACT || k < nc) c2[rp][k] = add2(c2[rp][k], M2);
                                        float d0, d1;
                                        upk(sub2(g2[k], c2[rp][k]), d0, d1);
                                        p2[k] = pk(ex2(d0), ex2(d1));
                                        S2 = add2(S2, p2[k]);
                                    }
                                    upk(S2, S0, S1);
                                }
                            }
                            const float inv0 = v0 ? rcp_approx(S0) : 0.f;
                            const float inv1 = v1 ? rcp_approx(S1) : 0.f;
                            const f2 inv2 = pk(inv0, inv1);
    #pragma unroll
                            for (int k = 0; k < NCB; ++k) cs2[k] = fma2(p2[k], inv2, cs2[k]);
                            if (last) {
                                float w0 = 0.f, w1 = 0.f;
    #pragma unroll
                                for (int k = 0; k < NCB; ++k) {
                                    if (k < a.K) {
                                        float p0, p1;
                                        upk(p2[k], p0, p1);
                                        w0 += s.e[k] * p0;
                                        w1 += s.e[k] * p1;
                                    }
                                }
                                acc_imp[2 * rp] += rr[2 * rp] * (w0 * inv0);
                                acc_imp[2 * rp + 1] += rr[2 * rp + 1] * (w1 * inv1);
                            }
                        }
                    };
                    if constexpr (EXPF_OK) {
                        if (__builtin_expect(lg, 0))
                            sweep(BoolTag<false>{});
                        else
                            sweep(BoolTag<true>{});
                    } else {
                        sweep(BoolTag<false>{});
                    }
                    float cs[NCB];
    #pragma unroll
                    for (int k = 0; k < NCB; ++k) {
                        float lo, hi;
                        upk(cs2[k], lo, hi);
                        cs[k] = lo + hi;
                    }
                    column_update<NCB, GPL, REC>(cs, gm, nc, s.red, s.ib, par, lane, warp, W,
                                                 REC ? a.gall + ((size_t)u * a.L + l) * nc : nullptr,
                                                 REC ? a.csall + ((size_t)u * a.L + l) * nc : nullptr);
                    par ^= 1;
                    if (l == 0 && tid == 0)
                        stage_consumer(na, nu, ncn, na.ld, s, MODE == MODE_UPDATE_SWEEP && a.optimizer == 0, false);
                };
                if constexpr (PEEL) {
                    for (int l = 0; l < a.L - 1; ++l) iteration(l, BoolTag<false>{});
                    iteration(a.L - 1, BoolTag<true>{});
                } else {
                    for (int l = 0; l < a.L; ++l) iteration(l, l == a.L - 1);
                }
            } else {
                auto iteration = [&](int l, auto tag) {
                    const bool last = last_of(tag);
                    if (last && warp == 0) {
    #pragma unroll
                        for (int j = 0; j < GPL; ++j)
                            if (j * 32 + lane < nc) a.gP[(size_t)u * nc + j * 32 + lane] = gm[j];
                    }
                    float gk[NCB];
                    bcast_g<NCB, GPL>(gm, gk);
                    float cs[NCB];
    #pragma unroll
                    for (int k = 0; k < NCB; ++k) cs[k] = 0.f;
    #pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (!vr[r]) continue;
                        float p[NCB];
                        float S = 0.f;
    #pragma unroll
                        for (int k = 0; k < NCB; ++k) {
                            p[k] = ex2(gk[k] - c[r][k]);
                            S += p[k];
                        }
                        if (!(S >= 0x1p-64f && S <= 0x1p64f)) {
                            float M = -INFINITY;
    #pragma unroll
                            for (int k = 0; k < NCB; ++k)
                                if (EXACT || k < nc) M = fmaxf(M, gk[k] - c[r][k]);
                            S = 0.f;
    #pragma unroll
                            for (int k = 0; k < NCB; ++k) {
                                if (EXACT || k < nc) c[r][k] += M;
                                p[k] = ex2(gk[k] - c[r][k]);
                                S += p[k];
                            }
                        }
                        const float inv = rcp_approx(S);
    #pragma unroll
                        for (int k = 0; k < NCB; ++k) cs[k] += p[k] * inv;
                        if (last) {
                            float v = 0.f;
    #pragma unroll
                            for (int k = 0; k < NCB; ++k)
                                if (k < a.K) v += s.e[k] * p[k];
                            acc_imp[r] += rr[r] * (v * inv);
                        }
                    }
                    column_update<NCB, GPL, REC>(cs, gm, nc, s.red, s.ib, par, lane, warp, W,
                                                 REC ? a.gall + ((size_t)u * a.L + l) * nc : nullptr,
                                                 REC ? a.csall + ((size_t)u * a.L + l) * nc : nullptr);
                    par ^= 1;
                    if (l == 0 && tid == 0)
                        stage_consumer(na, nu, ncn, na.ld, s, MODE == MODE_UPDATE_SWEEP && a.optimizer == 0, false);
                };
                if constexpr (PEEL) {
                    for (int l = 0; l < a.L - 1; ++l) iteration(l, BoolTag<false>{});
                    iteration(a.L - 1, BoolTag<true>{});
                } else {
                    for (int l = 0; l < a.L; ++l) iteration(l, l == a.L - 1);
                }
            }
            }  // register sweep
            if (warp == 0) {
    #pragma unroll
                for (int j = 0; j < GPL; ++j)
                    if (j * 32 + lane < nc) a.gL[(size_t)u * nc + j * 32 + lane] = gm[j];
            }
            // tile sweep: the last column update ended with a barrier after every read of the tile, so
            // the next consumer's tile can be staged now (its L2 prefetch was issued during the solve)
            if (TS && tid == 0) stage_consumer(na, nu, ncn, na.ld, s, false, TS);
    }
    return true;
}

// Shared arrays of market a that the consumers of a CTA read: exposure, 1 / b_k, omega (register
// sweep, update modes) and the Adam step size and bias correction of this step (t counts the steps
// applied before it). Made visible by the next barrier.
template <int NCB, bool EXACT, int MODE, int TS>
__device__ __forceinline__ void p1_market_setup(const P1Args& a, const Smem& s) {
    const int nc = EXACT ? NCB : a.nc;
    const int ncx = ncx_of(nc, NCB);
    const int tid = threadIdx.x, T = blockDim.x;
    if (tid == 0) {
        float step_size = a.lr, bc2s = 1.f;
        if (MODE == MODE_UPDATE_SWEEP && a.optimizer == 0) {
            const float t1 = (float)(a.st->t + 1);
            step_size = a.lr / one_minus_pow(a.beta1, t1);
            bc2s = sqrtf(one_minus_pow(a.beta2, t1));
        }
        s.coef[0] = step_size;
        s.coef[1] = bc2s;
    }
    for (int k = tid; k < ncx; k += T) {
        s.ib[k] = k < nc ? a.invb[k] : 0.f;
        s.e[k] = k < nc ? a.e[k] : 0.f;
    }
    if (MODE != MODE_SWEEP && !TS)
        for (int i = tid; i < a.ld; i += T) s.om[i] = i < a.I ? a.omega[i] : 0.f;
}

// Launch bound: 512 threads, except the tile sweep of more than 16 columns, which serves at most
// 2048 items (256 threads) and may then use up to 255 registers per thread.
template <int NCB, int R, bool EXACT, int MODE, int TS, bool REC = false>
__global__ void __launch_bounds__((TS != 0 && NCB > 16) ? 256 : 512) p1_kernel(const P1Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nc = EXACT ? NCB : a.nc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int ld = a.ld;
    const int i0 = tid * R;
    Smem s;
    smem_layout(NCB, nc, ld, W, MODE, TS, &s, smem_raw);

    if (a.st->stop) return;  // fr_solve reached its threshold: the remaining steps are no-ops

    // Staggered start of the ascent step. Every CTA alternates a gradient step (its Adam pass
    // streams the moments from HBM) and an on-chip Sinkhorn solve, and CTAs that start together
    // stay in phase, so their memory-bound phases coincide. CTAs in the upper half of the grid that
    // have fewer consumers than the busiest CTA (which sets the kernel's duration) start a quarter
    // of a consumer period late -- time they would otherwise spend idle at the end -- so that their
    // gradient steps fall into the other CTAs' solves (2000 x 1000 x 11: 4 % shorter step). The
    // period is CTA 0's time per consumer in the previous launch. Only the timing changes.
    const int n_mine = (a.U - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const int n_most = (a.U + (int)gridDim.x - 1) / (int)gridDim.x;
    unsigned long long t_launch = 0;
    if constexpr (MODE == MODE_UPDATE_SWEEP) {
        if (blockIdx.x == 0 && tid == 0) t_launch = global_ns();
        const unsigned long long period = a.st->cta_ns;
        if (n_mine < n_most && blockIdx.x >= gridDim.x / 2 && period > 0) {
            const unsigned long long t0 = global_ns(), delay = period / 4;
            for (int it = 0; it < 8192; ++it) {  // bounded: at most ~8 ms of 1 us naps
                if (global_ns() - t0 >= delay) break;
                __nanosleep(1000);
            }
        }
    }

    if (tid == 0) {
        mbar_init(s.bar, 1);
        fence_mbar_init();
    }
    __syncthreads();  // the mbarrier is initialised before any thread waits on it
    if (tid == 0)
        stage_consumer(a, blockIdx.x, nc, ld, s, MODE == MODE_UPDATE_SWEEP && a.optimizer == 0, TS);
    p1_market_setup<NCB, EXACT, MODE, TS>(a, s);

    float acc_imp[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc_imp[r] = 0.f;
    double gn2 = 0.0;
    int par = 0;
    unsigned phase = 0;

    for (int u = blockIdx.x; u < a.U; u += gridDim.x) {
        const int nu = u + (int)gridDim.x < a.U ? u + (int)gridDim.x : -1;
        if (!p1_consumer<NCB, R, EXACT, MODE, TS, REC>(a, s, u, a, nu, a.part + (size_t)blockIdx.x * ld,
                                                  u == (int)blockIdx.x, acc_imp, gn2, par, phase))
            break;
    }
    if constexpr (MODE != MODE_GRAD) {
        if constexpr (TS == 0) {  // (the tile sweep accumulates into part as it goes)
            if (i0 < ld) stv<R>(a.part + (size_t)blockIdx.x * ld + i0, acc_imp);
        }
    }
    if constexpr (MODE == MODE_UPDATE_SWEEP) {
        // CTA sum of the squared gradient in double, fixed order
        __syncthreads();
        double* s_d = reinterpret_cast<double*>(s.red);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gn2 += __shfl_xor_sync(FULL, gn2, o);
        if (lane == 0) s_d[warp] = gn2;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < W; ++w) t += s_d[w];
            a.gn2_part[blockIdx.x] = t;
            if (blockIdx.x == 0 && n_mine > 0) a.st->cta_ns = (global_ns() - t_launch) / n_mine;
        }
    }
}

// Batched markets: CTA b walks chunks b, b + G, ... of the list; a chunk is a run of consecutive
// consumers of one market with its own partial row (impacts, and the squared gradient in update
// mode). The chunk's market arguments are copied to shared memory; the tile of the next chunk's
// first consumer is staged during the previous chunk's last consumer, as in p1_kernel. One shared
// layout (the variant's at ld_max) serves every market of the launch.
template <int NCB, int R, bool EXACT, int MODE, int TS>
__global__ void __launch_bounds__((TS != 0 && NCB > 16) ? 256 : 512) p1_batch_kernel(const P1Batch bt) {
    static_assert(MODE != MODE_GRAD, "batched launches solve");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ P1Args sa;  // the current chunk's market
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int i0 = tid * R;
    Smem s;
    smem_layout(NCB, NCB, bt.ld_max, W, MODE, TS, &s, smem_raw);
    if ((int)blockIdx.x >= bt.n_chunks) return;
    if (tid == 0) {
        mbar_init(s.bar, 1);
        fence_mbar_init();
    }
    __syncthreads();  // the mbarrier is initialised before any thread waits on it
    if (tid == 0) {
        const P2Chunk c0 = bt.ch[blockIdx.x];
        const P1Args& a0 = bt.mk[c0.market];
        stage_consumer(a0, c0.u0, EXACT ? NCB : a0.nc, a0.ld, s,
                       MODE == MODE_UPDATE_SWEEP && a0.optimizer == 0, TS);
    }
    float acc_imp[R];
    int par = 0;
    unsigned phase = 0;
    for (int c = blockIdx.x; c < bt.n_chunks; c += gridDim.x) {
        const P2Chunk ch = bt.ch[c];
        __syncthreads();  // every thread is done with the previous chunk's market arrays
        if (tid == 0) sa = bt.mk[ch.market];
        __syncthreads();
        const P1Args& a = sa;
        p1_market_setup<NCB, EXACT, MODE, TS>(a, s);
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) acc_imp[r] = 0.f;
        double gn2 = 0.0;
        const int cn = c + (int)gridDim.x < bt.n_chunks ? c + (int)gridDim.x : -1;
        float* part_row = a.part + (size_t)ch.row * a.ld;
        bool ok = true;
        for (int u = ch.u0; u < ch.u1 && ok; ++u) {
            const P1Args* na = &a;
            int nu = u + 1;
            if (nu >= ch.u1) {
                if (cn >= 0) {
                    const P2Chunk nx = bt.ch[cn];
                    na = bt.mk + nx.market;
                    nu = nx.u0;
                } else {
                    nu = -1;
                }
            }
            ok = p1_consumer<NCB, R, EXACT, MODE, TS>(a, s, u, *na, nu, part_row, u == ch.u0, acc_imp,
                                                      gn2, par, phase);
        }
        if (!ok) break;  // an expired wait (the same in every thread): the CTA stops
        if constexpr (TS == 0) {
            if (i0 < a.ld) stv<R>(part_row + i0, acc_imp);
        }
        if constexpr (MODE == MODE_UPDATE_SWEEP) {  // the chunk's squared gradient, fixed order
            __syncthreads();
            double* s_d = reinterpret_cast<double*>(s.red);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) gn2 += __shfl_xor_sync(FULL, gn2, o);
            if (lane == 0) s_d[warp] = gn2;
            __syncthreads();
            if (tid == 0) {
                double t = 0.0;
                for (int w = 0; w < W; ++w) t += s_d[w];
                a.gn2_part[ch.row] = t;
            }
        }
    }
}

// Builds P1Variant entries: MkPlain with the single-market kernels (fn), MkBatch with the batched
// ones (fb). One variant table (p1_select_with) serves both.
struct MkPlain {
    template <int NCB, int R, bool EXACT, int TS>
    P1Variant make(int threads) const;
};
struct MkBatch {
    template <int NCB, int R, bool EXACT, int TS>
    P1Variant make(int threads) const {
        P1Variant v{};
        v.ncb = NCB;
        v.rows = R;
        v.exact = EXACT;
        v.threads = threads;
        v.tile_stride = TS;
        v.fb[0] = (const void*)p1_batch_kernel<NCB, R, EXACT, MODE_SWEEP, TS>;
        v.fb[1] = (const void*)p1_batch_kernel<NCB, R, EXACT, MODE_UPDATE_SWEEP, TS>;
        return v;
    }
};

// TS: 0 register sweep, else the tile sweep with that shared column stride (floats)
template <int NCB, int R, bool EXACT, int TS = 0>
P1Variant make_variant(int threads) {
    P1Variant v{};
    v.ncb = NCB;
    v.rows = R;
    v.exact = EXACT;
    v.threads = threads;
    v.smem = 0;
    v.tile_stride = TS;
    v.fn[MODE_SWEEP] = (const void*)p1_kernel<NCB, R, EXACT, MODE_SWEEP, TS>;
    v.fn[MODE_UPDATE_SWEEP] = (const void*)p1_kernel<NCB, R, EXACT, MODE_UPDATE_SWEEP, TS>;
    v.fn[MODE_GRAD] = (const void*)p1_kernel<NCB, R, EXACT, MODE_GRAD, TS>;
    v.fn_rec = (const void*)p1_kernel<NCB, R, EXACT, MODE_SWEEP, TS, true>;
    return v;
}

template <int NCB, int R, bool EXACT, int TS>
P1Variant MkPlain::make(int threads) const {
    return make_variant<NCB, R, EXACT, TS>(threads);
}

// 21 columns (20 slots + dummy): the tile sweep with eight rows per thread, at a shared column
// stride of 512, 1024 or 2048 floats.
template <class Mk>
bool p1_k21_with(const Mk& mk, int ld, int threads, P1Variant* out) {
    if (ld <= 512)
        *out = mk.template make<21, 8, true, 512>(threads);
    else if (ld <= 1024)
        *out = mk.template make<21, 8, true, 1024>(threads);
    else if (ld <= 2048)
        *out = mk.template make<21, 8, true, 2048>(threads);
    else
        return false;
    return true;
}

// Compiled variants: exact column counts for the hot shapes, padded buckets for the rest. k21 builds
// the 21-column entries (compiled in their own translation units).
template <class Mk>
bool p1_select_with(const Mk& mk, int nc, int I, P1Variant* out,
                    bool (*k21)(int ld, int threads, P1Variant* out)) {
    // CTA size: one thread per R items, at most 512 threads (the kernels' launch bound)
    auto threads_for = [&](int R) {
        int t = (I + R - 1) / R;
        return (t + 31) / 32 * 32;
    };
    P1Variant v;
    // 11 columns: costs in registers up to 768 items; beyond that the tile sweep (eight rows per
    // thread, costs read from the resident tile at a compile-time column stride of 1024, 2048 or
    // 4096 floats), up to 4096 items. Measured fused steps: 2000 x 1000 0.485 vs 0.506 ms,
    // 2000 x 2000 0.977 vs 1.126 ms, 250 x 2000 0.148 vs 0.174 ms for the tile sweep; at 250 and
    // 500 items a 1024-float stride leaves one-warp CTAs four to an SM and the tile sweep runs
    // at half the register sweep's speed.
    const int ld = (I + 7) / 8 * 8;
    if (nc == 11 && ld <= 768 && threads_for(4) <= 512) {
        v = mk.template make<11, 4, true, 0>(threads_for(4));
    } else if (nc == 11 && threads_for(8) <= 512) {
        if (ld <= 1024)
            v = mk.template make<11, 8, true, 1024>(threads_for(8));
        else if (ld <= 2048)
            v = mk.template make<11, 8, true, 2048>(threads_for(8));
        else
            v = mk.template make<11, 8, true, 4096>(threads_for(8));
    } else if (nc == 21 && threads_for(8) <= 256 && k21(ld, threads_for(8), &v)) {
        // 21 columns: the tile sweep (exact, eight rows per thread, at most 256 threads) up to
        // 2048 items
    } else if (nc == 50 && threads_for(1) <= 512) {
        v = mk.template make<50, 1, true, 0>(threads_for(1));
    } else if (nc <= 8 && threads_for(4) <= 512) {
        v = mk.template make<8, 4, false, 0>(threads_for(4));
    } else if (nc <= 16 && threads_for(4) <= 512) {
        v = mk.template make<16, 4, false, 0>(threads_for(4));
    } else if (nc <= 32 && threads_for(2) <= 512) {
        v = mk.template make<32, 2, false, 0>(threads_for(2));
    } else if (nc <= 64 && threads_for(1) <= 512) {
        v = mk.template make<64, 1, false, 0>(threads_for(1));
    } else {
        return false;
    }
    *out = v;
    return true;
}

}  // namespace

}  // namespace fr
