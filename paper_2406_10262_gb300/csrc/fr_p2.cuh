// fr_p2.cuh -- kernels of the per-item parametrisation c_uik = -r(u,i) e_k exp(theta_i).
//
// The costs are never stored: a row's costs are regenerated from one scalar per row and pass,
//   s_i = r(u,i) w_i / (eps ln 2),  w_i = exp(theta_i),
// so in log2 units x_ik = softmax_k(g'_k + s_i e_k). Shifting each row by s_i * max_k e_k (a row
// shift the Sinkhorn row update absorbs) gives the exponent g'_k + s_i (e_k - e_max) with
// e_k - e_max <= 0: one FMA and one exp2 per cell, computed two columns at a time with packed
// f32x2 FMAs. The column potentials are re-referenced to the last column after every column update
// (a common shift of g' leaves x unchanged), which keeps the exponents bounded.
//
// A thread owns R consecutive items of the consumer; with one scalar per row R can be 8 to 24, so
// the per-iteration column reduction (warp reduce-scatter, one CTA barrier) is amortised over
// R * m cells per thread. The relevance row of the next consumer is bulk-copied (TMA) into the
// other half of a double buffer during the current consumer's iterations; relevance is FP32 or
// BF16 (converted to FP32 on load; all arithmetic is FP32).
//
// p2_sweep_kernel: L Sinkhorn iterations per consumer (Problem (7)), emitting the policy of the
//   last row update; impact contributions r(u,i) sum_{k<K} e_k x_ik (Eq. 4) accumulate per CTA in
//   shared memory and are written to part[blockIdx][i] once per launch.
// p2_grad_kernel: gradient of L = sum_i omega_i Imp_i at the current policy by implicit
//   differentiation of the optimality conditions of Problem (7) (the same (m-1) x (m-1) system as
//   the free-cost path), reduced onto theta through dc_ik/dtheta_i = -r(u,i) e_k w_i:
//     dL/dtheta_i += (r w / eps) rho_i,  dL/dr(u,i) = omega_i v_i + (w / eps) rho_i,
//     rho_i = sum_k e_k x_ik (G_ik - alpha_i - beta_k),  v_i = sum_{k<K} e_k x_ik,
//   with per-CTA shared accumulators of dL/dtheta written to part[blockIdx][i].
#pragma once
#include <cuda_bf16.h>

#include "fr_device.cuh"
#include "fr_internal.h"

namespace fr {
namespace p2 {

__host__ __device__ inline int ncp(int nc) { return (nc + 3) / 4 * 4; }
__host__ __device__ inline int ncx(int nc, int ncb) { return ncp(nc > ncb ? nc : ncb); }

// Triangular index of Gram entry (k, l), k <= l < ncb-1.
__host__ __device__ constexpr int tri(int ncb, int k, int l) {
    return k * (ncb - 1) - k * (k - 1) / 2 + (l - k);
}
// End of the Gram pass that starts at row kb: as many rows as fit in `cap` accumulators.
__host__ __device__ constexpr int gram_end(int ncb, int kb, int cap) {
    int ke = kb + 1;
    while (ke < ncb - 1 && tri(ncb, ke + 1, ke + 1) - tri(ncb, kb, kb) <= cap) ++ke;
    return ke;
}
constexpr int GRAM_CAP = 56;

struct SweepSmem {
    float* w;     // [ld] exp(theta)
    float* acc;   // [ld] per-CTA impact partials
    unsigned char* rbuf;  // [2][ld] staged relevance rows (float or bf16)
    float* e;     // [ncx]
    float* eh;    // [ncx] e_k - e_max (0 beyond nc)
    float* ib;    // [ncx] 1 / b_k
    float* red;   // [2 * W * P]
    unsigned long long* bar;  // [2]
};

__host__ __device__ inline size_t sweep_layout(int ncb, int nc, int ld, int W, int esz,
                                               SweepSmem* s, unsigned char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 15) / 16 * 16;
        return o;
    };
    const int P = pow2ceil(ncb), nx = ncx(nc, ncb);
    const size_t o_bar = take(2 * sizeof(unsigned long long));
    const size_t o_w = take(sizeof(float) * ld), o_acc = take(sizeof(float) * ld);
    const size_t o_rb = take((size_t)2 * esz * ld);
    const size_t o_e = take(sizeof(float) * nx), o_eh = take(sizeof(float) * nx);
    const size_t o_ib = take(sizeof(float) * nx);
    const size_t o_red = take(sizeof(float) * 2 * W * P);
    if (s) {
        s->bar = (unsigned long long*)(base + o_bar);
        s->w = (float*)(base + o_w);
        s->acc = (float*)(base + o_acc);
        s->rbuf = base + o_rb;
        s->e = (float*)(base + o_e);
        s->eh = (float*)(base + o_eh);
        s->ib = (float*)(base + o_ib);
        s->red = (float*)(base + o_red);
    }
    return off;
}

__device__ __forceinline__ float load_r(const unsigned char* buf, int i, bool bf16) {
    return bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(buf)[i])
                : reinterpret_cast<const float*>(buf)[i];
}

// Thread 0: bulk copy of consumer un's relevance row into staging buffer b (of two).
__device__ __forceinline__ void p2_stage(const P2Args& a, int un, int b, unsigned long long* bars,
                                         unsigned char* rbuf, int esz) {
    if (un >= a.U) return;
    const unsigned bytes = (unsigned)((size_t)esz * a.ld);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(bars + b, bytes);
    bulk_g2s(rbuf + (size_t)b * esz * a.ld,
             static_cast<const unsigned char*>(a.r) + (size_t)un * esz * a.ld, bytes, bars + b);
}

// One row of the policy in base 2: p_k = 2^(g'_k + s (e_k - e_max)) for the column pairs (p2) and
// the unpaired last column (pt); returns 1 / sum_k p_k. A row whose sum leaves [2^-100, 2^100] is
// recomputed with its exact maximum subtracted, the maximum taken over the same packed exponents
// (padding columns carry g' = -inf there), so the scalar potentials need not stay live.
template <int NCB, bool EXACT>
__device__ __forceinline__ float p2_row(float sv, const f2* e2, float et, const f2* g2, float gt,
                                        const float* eh, const float (&gk)[NCB], int nc, f2* p2,
                                        float& pt) {
    constexpr int NP = NCB / 2;
    constexpr bool TAIL = NCB % 2 == 1;
    const f2 sp = pk(sv, sv);
    f2 S2 = 0ull;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        float a0, a1;
        upk(fma2(sp, e2[j], g2[j]), a0, a1);
        p2[j] = pk(ex2(a0), ex2(a1));
        S2 = add2(S2, p2[j]);
    }
    pt = TAIL ? ex2(fmaf(sv, et, gt)) : 0.f;
    float S0, S1;
    upk(S2, S0, S1);
    float S = S0 + S1 + pt;
    if (__builtin_expect(!(S >= 0x1p-100f && S <= 0x1p100f), 0)) {  // exact max shift for this row
        float M = TAIL ? fmaf(sv, et, gt) : -INFINITY;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            float a0, a1;
            upk(fma2(sp, e2[j], g2[j]), a0, a1);
            M = fmaxf(M, fmaxf(a0, a1));
        }
        S2 = 0ull;
        const f2 M2 = pk(M, M);
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            float a0, a1;
            upk(sub2(fma2(sp, e2[j], g2[j]), M2), a0, a1);
            p2[j] = pk(ex2(a0), ex2(a1));
            S2 = add2(S2, p2[j]);
        }
        pt = TAIL ? ex2(fmaf(sv, et, gt) - M) : 0.f;
        upk(S2, S0, S1);
        S = S0 + S1 + pt;
    }
    return rcp_approx(S);
}

// Column sums of per-thread vectors over the CTA, delivered to every warp: lane l of every warp
// gets the sums of columns l, l+32, ... (fixed order). One __syncthreads on buffer `par`.
template <int NCB, int GPL>
__device__ __forceinline__ void column_sum(float (&cs)[NCB], float (&out)[GPL], int nc,
                                           float* s_red, int par, int lane, int warp, int W) {
    constexpr int P = pow2ceil(NCB);
    constexpr int PER = P >= 32 ? P / 32 : 1;
    float w[P];
#pragma unroll
    for (int k = 0; k < P; ++k) w[k] = k < NCB ? cs[k] : 0.f;
    bool owner;
    const int base = warp_reduce_scatter<P>(w, lane, owner);
    float* buf = s_red + (size_t)par * W * P;
    if (owner) {
#pragma unroll
        for (int q = 0; q < PER; ++q)
            if (base + q < nc) buf[warp * P + base + q] = w[q];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
        const int col = j * 32 + lane;
        float sum = 0.f;
        if (col < nc)
            for (int ww = 0; ww < W; ++ww) sum += buf[ww * P + col];
        out[j] = sum;
    }
}

// One Sinkhorn iteration of one consumer (LAST: also the policy's impact contributions and gP).
template <int NCB, int R, bool EXACT, bool LAST>
__device__ __forceinline__ void sweep_iter(const P2Args& a, const SweepSmem& s, int l, int u,
                                           int u_step, int u_end, int b, int esz, bool bf16,
                                           const unsigned char* rrow, const f2* e2, float et,
                                           const float (&sv)[R], const bool (&vr)[R],
                                           float (&gm)[(NCB + 31) / 32], int& par, int i0, int nc,
                                           int lane, int warp, int W, int tid) {
    constexpr int GPL = (NCB + 31) / 32;
    constexpr int NP = NCB / 2;
    constexpr bool TAIL = NCB % 2 == 1;
    const int ref = nc - 1;
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < GPL; ++j) {
            const int col = j * 32 + lane;
            if (col >= nc) continue;
            if (LAST) a.gP[(size_t)u * nc + col] = gm[j];
            if (a.ck && l % a.ce == 0)  // g^(l), the start of segment l / ce
                a.ck[((size_t)u * a.nck + l / a.ce) * nc + col] = gm[j];
        }
    }
    float gk[NCB];
    bcast_g<NCB, GPL>(gm, gk);
    if (!EXACT) {
#pragma unroll
        for (int k = 0; k < NCB; ++k)
            if (k >= nc) gk[k] = -INFINITY;  // padding columns: 2^(-inf) = 0
    }
    f2 g2[NP > 0 ? NP : 1];
#pragma unroll
    for (int j = 0; j < NP; ++j) g2[j] = pk(gk[2 * j], gk[2 * j + 1]);
    const float gt = TAIL ? gk[NCB - 1] : 0.f;
    f2 cs2[NP > 0 ? NP : 1];
#pragma unroll
    for (int j = 0; j < NP; ++j) cs2[j] = 0ull;
    float cst = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (!vr[r]) continue;
        f2 p2[NP > 0 ? NP : 1];
        float pt;
        const float inv = p2_row<NCB, EXACT>(sv[r], e2, et, g2, gt, s.eh, gk, nc, p2, pt);
        const f2 inv2 = pk(inv, inv);
#pragma unroll
        for (int j = 0; j < NP; ++j) cs2[j] = fma2(p2[j], inv2, cs2[j]);
        cst = fmaf(pt, inv, cst);
        if (LAST) {
            float v = 0.f;
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                float p0, p1;
                upk(p2[j], p0, p1);
                if (2 * j < a.K) v += s.e[2 * j] * p0;
                if (2 * j + 1 < a.K) v += s.e[2 * j + 1] * p1;
            }
            if (TAIL && NCB - 1 < a.K) v += s.e[NCB - 1] * pt;
            s.acc[i0 + r] += load_r(rrow, i0 + r, bf16) * (v * inv);
        }
    }
    float cs[NCB];
#pragma unroll
    for (int j = 0; j < NP; ++j) upk(cs2[j], cs[2 * j], cs[2 * j + 1]);
    if (TAIL) cs[NCB - 1] = cst;
    // column sums (the reduction of column_update, written out here so that they can be kept
    // for the adjoint), then g'_k -= log2(cs_k / b_k)
    float csum[GPL];
    column_sum<NCB, GPL>(cs, csum, nc, s.red, par, lane, warp, W);
    par ^= 1;
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
        const int col = j * 32 + lane;
        if (col < nc) {
            gm[j] -= log2_near1(fmaxf(csum[j] * s.ib[col], 1e-37f));
            if (a.csk && warp == 0) a.csk[((size_t)u * a.L + l) * nc + col] = csum[j];
        }
    }
    // re-reference the potentials to the last column (x is invariant to a common shift)
    const float gref = __shfl_sync(FULL, gm[ref / 32], ref % 32);
#pragma unroll
    for (int j = 0; j < GPL; ++j) gm[j] -= gref;
    if (l == 0 && tid == 0 && u + u_step < u_end) p2_stage(a, u + u_step, b ^ 1, s.bar, s.rbuf, esz);
}

// Sinkhorn sweep of consumers u_first, u_first + u_step, ... < u_end of one market (one CTA), impact
// partials of those consumers written to part_row[0 .. ld). Staging buffer index b, the mbarrier
// phase bits and the reduction buffer parity carry over between calls of one CTA.
template <int NCB, int R, bool EXACT>
__device__ __forceinline__ void sweep_consumers(const P2Args& a, int u_first, int u_end, int u_step,
                                                float* __restrict__ part_row, const SweepSmem& s,
                                                int& b, unsigned& phase_bits, int& par) {
    constexpr int GPL = (NCB + 31) / 32;
    constexpr int NP = NCB / 2;         // column pairs
    constexpr bool TAIL = NCB % 2 == 1;  // one unpaired last column
    const int nc = EXACT ? NCB : a.nc;
    const int nx = ncx(nc, NCB);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int T = blockDim.x;
    const int I = a.I, ld = a.ld;
    const int i0 = tid * R;
    const bool bf16 = a.r_bf16 != 0;
    const int esz = bf16 ? 2 : 4;

    if (tid == 0) p2_stage(a, u_first, b, s.bar, s.rbuf, esz);
    for (int i = tid; i < ld; i += T) s.w[i] = i < I ? a.w[i] : 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (i0 + r < ld) s.acc[i0 + r] = 0.f;
    for (int k = tid; k < nx; k += T) {
        s.e[k] = k < nc ? a.e[k] : 0.f;
        s.eh[k] = k < nc ? a.e[k] - a.emax : 0.f;
        s.ib[k] = k < nc ? a.invb[k] : 0.f;
    }
    __syncthreads();
    // packed (e_k - e_max) pairs, constant for the market
    f2 e2[NP > 0 ? NP : 1];
#pragma unroll
    for (int j = 0; j < NP; ++j) e2[j] = pk(s.eh[2 * j], s.eh[2 * j + 1]);
    const float et = TAIL ? s.eh[NCB - 1] : 0.f;
    const int ref = nc - 1;  // gauge column
    bool vr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) vr[r] = i0 + r < I;

    for (int u = u_first; u < u_end; u += u_step, b ^= 1) {
        // the consumer's relevance row is the only copy in flight; if the bounded wait expires,
        // the CTA records a timeout, waits (default bound) for the copy to land and stops
        const bool row_ok = cta_wait_or_drain(s.bar + b, (phase_bits >> b) & 1u, a.max_polls,
                                              kDefaultPolls, &a.st->err, 4);
        phase_bits ^= 1u << b;
        if (!row_ok) break;
        const unsigned char* rrow = s.rbuf + (size_t)b * esz * ld;
        float sv[R];
#pragma unroll
        for (int r = 0; r < R; ++r)
            sv[r] = vr[r] ? load_r(rrow, i0 + r, bf16) * s.w[i0 + r] * a.inv_eps_ln2 : 0.f;
        float gm[GPL];
#pragma unroll
        for (int j = 0; j < GPL; ++j) {
            const int col = j * 32 + lane;
            gm[j] = (a.warm && col < nc) ? a.gL[(size_t)u * nc + col] : 0.f;
        }
        for (int l = 0; l < a.L - 1; ++l)
            sweep_iter<NCB, R, EXACT, false>(a, s, l, u, u_step, u_end, b, esz, bf16, rrow, e2, et, sv,
                                             vr, gm, par, i0, nc, lane, warp, W, tid);
        sweep_iter<NCB, R, EXACT, true>(a, s, a.L - 1, u, u_step, u_end, b, esz, bf16, rrow, e2, et,
                                        sv, vr, gm, par, i0, nc, lane, warp, W, tid);
        if (warp == 0) {
#pragma unroll
            for (int j = 0; j < GPL; ++j)
                if (j * 32 + lane < nc) a.gL[(size_t)u * nc + j * 32 + lane] = gm[j];
        }
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (i0 + r < ld) part_row[i0 + r] = s.acc[i0 + r];
    __syncthreads();  // shared arrays and the idle staging buffer are free for the next call
}

// Single market: CTA g sweeps consumers g, g + G, ... and writes partial row g.
template <int NCB, int R, bool EXACT>
__global__ void __launch_bounds__(512) p2_sweep_kernel(const P2Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SweepSmem s;
    sweep_layout(NCB, EXACT ? NCB : a.nc, a.ld, blockDim.x >> 5, a.r_bf16 ? 2 : 4, &s, smem_raw);
    if (a.st->stop) return;
    if (threadIdx.x == 0) {
        mbar_init(s.bar, 1);
        mbar_init(s.bar + 1, 1);
        fence_mbar_init();
    }
    __syncthreads();  // mbarriers initialised before any wait
    int par = 0, b = 0;
    unsigned phase_bits = 0u;  // bit b: expected phase parity of staging buffer b
    sweep_consumers<NCB, R, EXACT>(a, blockIdx.x, a.U, gridDim.x, a.part + (size_t)blockIdx.x * a.ld,
                                   s, b, phase_bits, par);
}

// Batched markets: CTA g takes chunks g, g + G, ... of the launch's chunk list, each a range of
// consumers of one market with its own partial row. The chunk's market arguments are staged in
// shared memory and read from there.
template <int NCB, int R, bool EXACT>
__global__ void __launch_bounds__(512) p2_sweep_batch_kernel(const P2Batch bt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ P2Args s_args;
    SweepSmem s;
    sweep_layout(NCB, NCB, bt.ld_max, blockDim.x >> 5, bt.esz, &s, smem_raw);
    if (threadIdx.x == 0) {
        mbar_init(s.bar, 1);
        mbar_init(s.bar + 1, 1);
        fence_mbar_init();
    }
    __syncthreads();  // mbarriers initialised before any wait
    int par = 0, b = 0;
    unsigned phase_bits = 0u;
    for (int c = blockIdx.x; c < bt.n_chunks; c += gridDim.x) {
        const P2Chunk ch = bt.ch[c];
        if (threadIdx.x == 0) s_args = bt.mk[ch.market];
        __syncthreads();
        if (!s_args.st->stop)
            sweep_consumers<NCB, R, EXACT>(s_args, ch.u0, ch.u1, 1,
                                           s_args.part + (size_t)ch.row * s_args.ld, s, b,
                                           phase_bits, par);
        __syncthreads();  // s_args is rewritten for the next chunk
    }
}

// ---- implicit gradient -------------------------------------------------------------------------
struct GradSmem {
    float* acc;    // [ld] per-CTA dL/dtheta partials
    float* lse;    // [ld]
    float* h;      // [ld]
    unsigned char* rbuf;  // [2][ld]
    float* e;      // [ncx]
    float* eh;     // [ncx]
    float* gp;     // [ncx]
    float* beta;   // [ncx]
    float* out;    // [3*ncp + NGALL]
    float* red;    // [W * max(3P, 64)]
    float* A;      // [n*n]
    float* rhs;    // [ncp]
    float* Lt;     // [n*n]
    unsigned long long* bar;  // [2]
};

__host__ __device__ inline size_t grad_layout(int ncb, int nc, int ld, int W, int esz, GradSmem* s,
                                              unsigned char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 15) / 16 * 16;
        return o;
    };
    const int P = pow2ceil(ncb), nx = ncx(nc, ncb), np = ncp(nc), n = nc - 1;
    const int NGALL = ncb * (ncb - 1) / 2;
    size_t red_f = (size_t)W * 3 * P;
    if ((size_t)W * 64 > red_f) red_f = (size_t)W * 64;
    const size_t o_bar = take(2 * sizeof(unsigned long long));
    const size_t o_acc = take(sizeof(float) * ld);
    const size_t o_lse = take(sizeof(float) * ld), o_h = take(sizeof(float) * ld);
    const size_t o_rb = take((size_t)2 * esz * ld);
    const size_t o_e = take(sizeof(float) * nx), o_eh = take(sizeof(float) * nx);
    const size_t o_gp = take(sizeof(float) * nx), o_beta = take(sizeof(float) * nx);
    const size_t o_out = take(sizeof(float) * (3 * np + NGALL));
    const size_t o_red = take(sizeof(float) * red_f);
    const size_t o_A = take(sizeof(float) * (size_t)(n > 0 ? n * n : 1));
    const size_t o_rhs = take(sizeof(float) * np);
    const size_t o_Lt = take(sizeof(float) * (size_t)(n > 0 ? n * n : 1));
    if (s) {
        s->bar = (unsigned long long*)(base + o_bar);
        s->acc = (float*)(base + o_acc);
        s->lse = (float*)(base + o_lse);
        s->h = (float*)(base + o_h);
        s->rbuf = base + o_rb;
        s->e = (float*)(base + o_e);
        s->eh = (float*)(base + o_eh);
        s->gp = (float*)(base + o_gp);
        s->beta = (float*)(base + o_beta);
        s->out = (float*)(base + o_out);
        s->red = (float*)(base + o_red);
        s->A = (float*)(base + o_A);
        s->rhs = (float*)(base + o_rhs);
        s->Lt = (float*)(base + o_Lt);
    }
    return off;
}

// One pass of the Gram accumulation over rows (rows strided over the CTA) for first indices
// k in [KB, KE), then the CTA reduction into gout[tri(k, l)]; recurses until the triangle is done.
template <int NCB, bool EXACT, int KB>
__device__ __forceinline__ void gram_passes(const GradSmem& s, const P2Args& a,
                                            const unsigned char* rrow, bool bf16, int nc,
                                            float* gout) {
    const int I = a.I;
    if constexpr (KB < NCB - 1) {
        constexpr int KE = gram_end(NCB, KB, GRAM_CAP);
        constexpr int N0 = tri(NCB, KB, KB);
        constexpr int NH = tri(NCB, KE, KE) - N0;
        const int n = nc - 1;
        float gram[NH];
#pragma unroll
        for (int q = 0; q < NH; ++q) gram[q] = 0.f;
        for (int i = threadIdx.x; i < I; i += blockDim.x) {
            const float si = load_r(rrow, i, bf16) * __ldg(a.w + i) * a.inv_eps_ln2;
            const float li = s.lse[i];
            float x[NCB];
#pragma unroll
            for (int k = KB; k < NCB; ++k)
                x[k] = (EXACT || k < nc) ? ex2(fmaf(si, s.eh[k], s.gp[k]) - li) : 0.f;
            int q = 0;
#pragma unroll
            for (int k = KB; k < KE; ++k) {
#pragma unroll
                for (int m = k; m < NCB - 1; ++m, ++q)
                    if (EXACT || m < n) gram[q] += k == m ? x[k] * (1.f - x[k]) : -x[k] * x[m];
            }
        }
        cta_reduce_vec<NH>(gram, NH, s.red, gout + N0);
        gram_passes<NCB, EXACT, KE>(s, a, rrow, bf16, nc, gout);
    }
}

// Implicit gradient of consumers u_first, u_first + u_step, ... < u_end of one market (one CTA);
// dL/dtheta partials of those consumers written to part_row[0 .. ld).
template <int NCB, bool EXACT>
__device__ __forceinline__ void grad_consumers(const P2Args& a, int u_first, int u_end, int u_step,
                                               float* __restrict__ part_row, const GradSmem& s,
                                               int& b, unsigned& phase_bits) {
    const int nc = EXACT ? NCB : a.nc;
    const int np_ = ncp(nc), nx = ncx(nc, NCB), n = nc - 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int T = blockDim.x;
    const int I = a.I, ld = a.ld;
    const bool bf16 = a.r_bf16 != 0;
    const int esz = bf16 ? 2 : 4;

    if (tid == 0) p2_stage(a, u_first, b, s.bar, s.rbuf, esz);
    for (int i = tid; i < ld; i += T) s.acc[i] = 0.f;
    for (int k = tid; k < nx; k += T) {
        s.e[k] = k < nc ? a.e[k] : 0.f;
        s.eh[k] = k < nc ? a.e[k] - a.emax : 0.f;
    }
    for (int u = u_first; u < u_end; u += u_step, b ^= 1) {
        // the consumer's relevance row is the only copy in flight; if the bounded wait expires,
        // the CTA records a timeout, waits (default bound) for the copy to land and stops
        const bool row_ok = cta_wait_or_drain(s.bar + b, (phase_bits >> b) & 1u, a.max_polls,
                                              kDefaultPolls, &a.st->err, 4);
        phase_bits ^= 1u << b;
        if (!row_ok) break;
        const unsigned char* rrow = s.rbuf + (size_t)b * esz * ld;
        for (int k = tid; k < nx; k += T) s.gp[k] = k < nc ? a.gP[(size_t)u * nc + k] : -INFINITY;
        __syncthreads();
        // pass A: policy rows, row normalisers, h, and the column sums q, cs, X^T h
        {
            float acc[3][NCB];
#pragma unroll
            for (int k = 0; k < NCB; ++k) acc[0][k] = acc[1][k] = acc[2][k] = 0.f;
            for (int i = tid; i < I; i += T) {
                const float ri = load_r(rrow, i, bf16);
                const float si = ri * __ldg(a.w + i) * a.inv_eps_ln2;
                float x[NCB];
                float M = -INFINITY;
#pragma unroll
                for (int k = 0; k < NCB; ++k) {
                    x[k] = (EXACT || k < nc) ? fmaf(si, s.eh[k], s.gp[k]) : -INFINITY;
                    M = fmaxf(M, x[k]);
                }
                float S = 0.f;
#pragma unroll
                for (int k = 0; k < NCB; ++k) {
                    x[k] = ex2(x[k] - M);
                    S += x[k];
                }
                const float inv = rcp_approx(S);  // S in [1, m]: the row max contributes 1
                const float wr = __ldg(a.omega + i) * ri;  // dL/dx_ik = wr_i e_k (k < K)
                float hh = 0.f;
#pragma unroll
                for (int k = 0; k < NCB; ++k) {
                    x[k] *= inv;
                    if (k < a.K) hh += x[k] * (wr * s.e[k]);
                }
#pragma unroll
                for (int k = 0; k < NCB; ++k) {
                    if (k < a.K) acc[0][k] += x[k] * (wr * s.e[k]);
                    acc[1][k] += x[k];
                    acc[2][k] += x[k] * hh;
                }
                s.lse[i] = M + lg2_approx(S);
                s.h[i] = hh;
            }
            cta_reduce<NCB, 3>(acc, nc, s.red, s.out, np_);  // [q | cs | X^T h]
        }
        // Gram block of diag(cs) - X^T X in passes over the triangle, then the solve
        float* gout = s.out + 3 * np_;
        gram_passes<NCB, EXACT, 0>(s, a, rrow, bf16, nc, gout);
        for (int idx = tid; idx < n * n; idx += T) {
            int k = idx / n, m = idx % n;
            if (k > m) { const int t = k; k = m; m = t; }
            s.A[idx] = gout[tri(NCB, k, m)];
        }
        for (int k = tid; k < nx; k += T) {
            if (k < n) s.rhs[k] = s.out[k] - s.out[2 * np_ + k];
            s.beta[k] = 0.f;
        }
        __syncthreads();
        if (warp == 0) warp_cholesky_solve_f32<NCB - 1>(s.A, s.rhs, n, s.Lt, s.beta, lane);
        __syncthreads();
        // final pass: alpha, rho, dL/dtheta partials and dL/dr
        for (int i = tid; i < I; i += T) {
            const float ri = load_r(rrow, i, bf16);
            const float wi = __ldg(a.w + i), oi = __ldg(a.omega + i);
            const float si = ri * wi * a.inv_eps_ln2, li = s.lse[i];
            const float wr = oi * ri;
            float x[NCB];
            float sb = 0.f;
#pragma unroll
            for (int k = 0; k < NCB; ++k) {
                x[k] = (EXACT || k < nc) ? ex2(fmaf(si, s.eh[k], s.gp[k]) - li) : 0.f;
                sb += x[k] * s.beta[k];
            }
            const float alpha = s.h[i] - sb;
            float rho = 0.f, v = 0.f;
#pragma unroll
            for (int k = 0; k < NCB; ++k) {
                const float G = k < a.K ? wr * s.e[k] : 0.f;
                rho += s.e[k] * x[k] * (G - alpha - s.beta[k]);
                if (k < a.K) v += s.e[k] * x[k];
            }
            s.acc[i] += ri * wi * rho * a.inv_eps;
            if (a.dr) a.dr[(size_t)u * I + i] = oi * v + wi * rho * a.inv_eps;
        }
        __syncthreads();  // staging buffer b^1 and the row arrays are free for the next consumer
        if (tid == 0 && u + u_step < u_end) p2_stage(a, u + u_step, b ^ 1, s.bar, s.rbuf, esz);
    }
    for (int i = tid; i < ld; i += T) part_row[i] = s.acc[i];
    __syncthreads();  // shared arrays are free for the next call
}

// Launch structures as the sweep kernels: one market with CTA-strided consumers, or a chunk list.
template <int NCB, int R, bool EXACT>
__global__ void __launch_bounds__(512) p2_grad_kernel(const P2Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GradSmem s;
    grad_layout(NCB, EXACT ? NCB : a.nc, a.ld, blockDim.x >> 5, a.r_bf16 ? 2 : 4, &s, smem_raw);
    if (a.st->stop) return;
    if (threadIdx.x == 0) {
        mbar_init(s.bar, 1);
        mbar_init(s.bar + 1, 1);
        fence_mbar_init();
    }
    __syncthreads();  // mbarriers initialised before any wait
    int b = 0;
    unsigned phase_bits = 0u;
    grad_consumers<NCB, EXACT>(a, blockIdx.x, a.U, gridDim.x, a.part + (size_t)blockIdx.x * a.ld, s,
                               b, phase_bits);
}

template <int NCB, int R, bool EXACT>
__global__ void __launch_bounds__(512) p2_grad_batch_kernel(const P2Batch bt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ P2Args s_args;
    GradSmem s;
    grad_layout(NCB, NCB, bt.ld_max, blockDim.x >> 5, bt.esz, &s, smem_raw);
    if (threadIdx.x == 0) {
        mbar_init(s.bar, 1);
        mbar_init(s.bar + 1, 1);
        fence_mbar_init();
    }
    __syncthreads();  // mbarriers initialised before any wait
    int b = 0;
    unsigned phase_bits = 0u;
    for (int c = blockIdx.x; c < bt.n_chunks; c += gridDim.x) {
        const P2Chunk ch = bt.ch[c];
        if (threadIdx.x == 0) s_args = bt.mk[ch.market];
        __syncthreads();
        if (!s_args.st->stop)
            grad_consumers<NCB, EXACT>(s_args, ch.u0, ch.u1, 1,
                                       s_args.part + (size_t)ch.row * s_args.ld, s, b, phase_bits);
        __syncthreads();
    }
}

template <int NCB, int R, bool EXACT>
P2Variant p2_make(int threads) {
    P2Variant v{};
    v.ncb = NCB;
    v.rows = R;
    v.exact = EXACT;
    v.threads = threads;
    v.sweep = (const void*)p2_sweep_kernel<NCB, R, EXACT>;
    v.grad = (const void*)p2_grad_kernel<NCB, R, EXACT>;
    v.sweep_b = (const void*)p2_sweep_batch_kernel<NCB, R, EXACT>;
    v.grad_b = (const void*)p2_grad_batch_kernel<NCB, R, EXACT>;
    return v;
}

}  // namespace p2
}  // namespace fr
