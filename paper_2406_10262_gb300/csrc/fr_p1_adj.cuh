// fr_p1_adj.cuh -- unrolled gradient of the free-cost parametrisation (Problem (8), one cost c_uik
// per cell): the adjoint of the L Sinkhorn iterations of Problem (7) that produced the emitted
// policy, with respect to every c_uik, taken in reverse with the column potentials checkpointed.
//
// Forward map of one consumer (natural units; iteration l = 1..L, warm start g^(0) a constant):
//   P^(l)_ik = softmax_k((g^(l-1)_k - c_ik) / eps)                         row update (Eq. 1)
//   g^(l)_k  = g^(l-1)_k + eps (log b_k - log cs^(l)_k), cs^(l)_k = sum_i P^(l)_ik   (Eq. 2)
//   x = P^(L)                                                               the emitted policy
// Reverse sweep for L = sum_i omega_i Imp_i, dL/dx_ik = gx_ik = omega_i r(u,i) e_k (dummy e = 0):
//   output layer: h_i = sum_k x_ik gx_ik, dc_ik -= x_ik (gx_ik - h_i) / eps,
//                 gbar^(L-1)_k = sum_i x_ik (gx_ik - h_i) / eps
//   l = L-1 .. 1: gc_k = gbar^(l)_k / cs^(l)_k,  a_i = sum_k P^(l)_ik gc_k,
//                 dc_ik += P^(l)_ik (gc_k - a_i),  gbar^(l-1)_k = sum_i P^(l)_ik a_i
// (g^(l) depends on the row potentials f^(l) with weight -P/cs and on c with +P/cs; f^(l) depends on
// g^(l-1) with weight -P and on c with +P). This is the same reverse sweep as the per-item
// adjoint, but every cell keeps its own dc_ik (held in registers by the thread owning the row).
//
// Checkpoints: the sweep that produced the policy stored each consumer's starting potentials
// g^(0) (P1Args::g0). The kernel re-runs the forward from g^(0), keeping g^(j ce) for
// j = 0 .. ceil(L/ce)-1 in shared memory, then walks the segments backwards, recomputing each
// segment's g^(l-1) and cs^(l) (2 ce m floats of shared memory) before reversing it. The forward
// iterations use the log form with an exact row-max shift (one exp2 per cell). With a checkpoint
// every iteration (ce = 1) the sweep records g^(l-1) and cs^(l) of every iteration
// (P1Args::gall / csall, 2 L m floats per consumer) and the kernel only runs the reverse.
//
// Modes: ADJ_GRAD writes dL/dC in the public layout [u][i][k] and dL/dr = omega_i v_i (C does not
// depend on r); ADJ_STEP applies the optimiser to the consumer's costs with dF/dC (omega = 1/Imp)
// and writes C and the Adam moments back, adding the squared gradient to the CTA's norm partial.
#pragma once
#include "fr_p2.cuh"

namespace fr {
namespace p1adj {

enum { ADJ_GRAD = 0, ADJ_STEP = 1 };

struct Smem {
    unsigned long long* bar;  // mbarrier of the staged copies
    float* C;     // [nc][ld] the consumer's costs (natural units)
    float* r;     // [ld] its relevance row
    float* e;     // [ncx] exposure (0 for the dummy and beyond nc)
    float* ib;    // [ncx] 1 / b_k
    float* ck;    // [nck][ncp] g'^(j ce) of the forward (log2 units)
    float* gs;    // [ce][ncp] g'^(l-1) of the segment
    float* cs;    // [ce][ncp] cs^(l) of the segment
    float* red;   // [2][W][P] column-sum partials
    double* dred; // [W] squared-gradient partials
};

__host__ __device__ inline int ncp1(int nc) { return (nc + 3) / 4 * 4; }

__host__ __device__ inline size_t layout(int ncb, int nc, int ld, int W, int ce, int nck, Smem* s,
                                         unsigned char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 15) / 16 * 16;
        return o;
    };
    const int P = pow2ceil(ncb), np = ncp1(nc > ncb ? nc : ncb);
    const size_t o_bar = take(sizeof(unsigned long long));
    const size_t o_C = take(sizeof(float) * (size_t)nc * ld);
    const size_t o_r = take(sizeof(float) * ld);
    const size_t o_e = take(sizeof(float) * np), o_ib = take(sizeof(float) * np);
    const size_t o_ck = take(sizeof(float) * (size_t)nck * np);
    const size_t o_gs = take(sizeof(float) * (size_t)ce * np);
    const size_t o_cs = take(sizeof(float) * (size_t)ce * np);
    const size_t o_red = take(sizeof(float) * 2 * W * P);
    const size_t o_dred = take(sizeof(double) * W);
    if (s) {
        s->bar = (unsigned long long*)(base + o_bar);
        s->C = (float*)(base + o_C);
        s->r = (float*)(base + o_r);
        s->e = (float*)(base + o_e);
        s->ib = (float*)(base + o_ib);
        s->ck = (float*)(base + o_ck);
        s->gs = (float*)(base + o_gs);
        s->cs = (float*)(base + o_cs);
        s->red = (float*)(base + o_red);
        s->dred = (double*)(base + o_dred);
    }
    return off;
}

// Thread 0: bulk-copies consumer un's cost tile and relevance row into shared memory.
__device__ __forceinline__ void stage(const P1Args& a, int un, int nc, int ld, const Smem& s) {
    if (un >= a.U) return;
    const unsigned tile = (unsigned)(sizeof(float) * (size_t)nc * ld);
    const unsigned row = (unsigned)(sizeof(float) * ld);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(s.bar, tile + row);
    bulk_g2s(s.C, a.C + (size_t)un * nc * ld, tile, s.bar);
    bulk_g2s(s.r, a.r + (size_t)un * ld, row, s.bar);
}

// Row i's policy at column potentials gk (log2 units, -inf beyond nc): p[k] = softmax_k(gk_k -
// c_ik / (eps ln 2)) with an exact max shift.
template <int NCB, bool EXACT>
__device__ __forceinline__ void row_policy(const float* Cs, int ld, int i, int nc, float sc,
                                           const float (&gk)[NCB], float (&p)[NCB]) {
    float M = -INFINITY;
#pragma unroll
    for (int k = 0; k < NCB; ++k) {
        p[k] = (EXACT || k < nc) ? gk[k] - Cs[k * ld + i] * sc : -INFINITY;
        M = fmaxf(M, p[k]);
    }
    float S = 0.f;
#pragma unroll
    for (int k = 0; k < NCB; ++k) {
        p[k] = ex2(p[k] - M);
        S += p[k];
    }
    const float inv = 1.f / S;
#pragma unroll
    for (int k = 0; k < NCB; ++k) p[k] *= inv;
}


// One forward Sinkhorn iteration of the consumer in shared memory: gm (g', lane-distributed) is
// advanced from g'^(l-1) to g'^(l); csum receives cs^(l) (lane-distributed). Every thread of the
// CTA must call it (one barrier).
template <int NCB, int R, bool EXACT>
__device__ __forceinline__ void fwd_iter(const Smem& s, int ld, int nc, int i0, const bool (&vr)[R],
                                         float sc, float (&gm)[(NCB + 31) / 32],
                                         float (&csum)[(NCB + 31) / 32], int& par, int lane,
                                         int warp, int W) {
    constexpr int GPL = (NCB + 31) / 32;
    float gk[NCB];
    bcast_g<NCB, GPL>(gm, gk);
    float csv[NCB];
#pragma unroll
    for (int k = 0; k < NCB; ++k) csv[k] = 0.f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (!vr[r]) continue;
        float p[NCB];
        row_policy<NCB, EXACT>(s.C, ld, i0 + r, nc, sc, gk, p);
#pragma unroll
        for (int k = 0; k < NCB; ++k) csv[k] += p[k];
    }
    p2::column_sum<NCB, GPL>(csv, csum, nc, s.red, par, lane, warp, W);
    par ^= 1;
#pragma unroll
    for (int j = 0; j < GPL; ++j) {
        const int col = j * 32 + lane;
        if (col < nc) gm[j] -= log2f(fmaxf(csum[j] * s.ib[col], 1e-37f));
    }
}

// One CTA per consumer at a time (persistent over u = blockIdx.x, blockIdx.x + G, ...); a thread
// owns R consecutive rows and their dc in registers.
template <int NCB, int R, bool EXACT, int MODE>
__global__ void __launch_bounds__(256) p1_adj_kernel(const P1Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int GPL = (NCB + 31) / 32;
    const int nc = EXACT ? NCB : a.nc;
    const int np = ncp1(nc > NCB ? nc : NCB);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int T = blockDim.x;
    const int I = a.I, ld = a.ld, L = a.L, ce = a.ce, nck = a.nck;
    const float sc = a.inv_eps_ln2, inv_eps = a.inv_eps;
    const int i0 = tid * R;
    Smem s;
    layout(NCB, nc, ld, W, ce, nck, &s, smem_raw);
    if (a.st->stop) return;

    if (tid == 0) {
        mbar_init(s.bar, 1);
        fence_mbar_init();
    }
    for (int k = tid; k < np; k += T) {
        s.e[k] = k < nc ? a.e[k] : 0.f;
        s.ib[k] = k < nc ? a.invb[k] : 0.f;
    }
    __syncthreads();  // mbarrier initialised, exposure and marginals visible
    if (tid == 0) stage(a, blockIdx.x, nc, ld, s);
    // optimiser coefficients of this step (t counts the steps applied before it)
    float step_size = a.lr, inv_bc2s = 1.f;
    if (MODE == ADJ_STEP && a.optimizer == 0) {
        const float t1 = (float)(a.st->t + 1);
        step_size = a.lr / one_minus_pow(a.beta1, t1);
        inv_bc2s = 1.f / sqrtf(one_minus_pow(a.beta2, t1));
    }
    bool vr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) vr[r] = i0 + r < I;
    double gn2 = 0.0;
    int par = 0;
    unsigned phase = 0;

    for (int u = blockIdx.x; u < a.U; u += gridDim.x) {
        // the consumer's tile is the only copy in flight; an expired bounded wait drains it and
        // stops the CTA (FR_ETIMEOUT)
        const bool tile_ok = cta_wait_or_drain(s.bar, phase, a.max_polls, kDefaultPolls, &a.st->err, 4);
        phase ^= 1u;
        if (!tile_ok) break;

        // ---- forward from the solve's starting potentials, keeping g'^(j ce), j < nck
        float gm[GPL], csum[GPL];
#pragma unroll
        for (int j = 0; j < GPL; ++j) {
            const int col = j * 32 + lane;
            gm[j] = col < nc ? a.g0[(size_t)u * nc + col] : 0.f;
        }
        for (int l = 0; !a.gall; ++l) {  // gm = g'^(l); none with the sweep's records
            if (l % ce == 0 && warp == 0) {
#pragma unroll
                for (int j = 0; j < GPL; ++j)
                    if (j * 32 + lane < nc) s.ck[(l / ce) * np + j * 32 + lane] = gm[j];
            }
            if (l >= (nck - 1) * ce) break;
            fwd_iter<NCB, R, EXACT>(s, ld, nc, i0, vr, sc, gm, csum, par, lane, warp, W);
        }
        __syncthreads();  // checkpoints visible

        // ---- reverse, segment by segment
        float dc[R][NCB], vi[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            vi[r] = 0.f;
#pragma unroll
            for (int k = 0; k < NCB; ++k) dc[r][k] = 0.f;
        }
        float gb[GPL];  // adjoint of the column potentials (natural units), lane-distributed
#pragma unroll
        for (int j = 0; j < GPL; ++j) gb[j] = 0.f;
        for (int seg = nck - 1; seg >= 0; --seg) {
            const int l0 = seg * ce, l1 = min(l0 + ce, L);
#pragma unroll
            for (int j = 0; j < GPL; ++j) {
                const int col = j * 32 + lane;
                gm[j] = col < nc ? s.ck[seg * np + col] : 0.f;
            }
            for (int l = l0 + 1; a.gall && l <= l1; ++l) {  // the sweep recorded them
                const int q = l - l0 - 1;
                if (warp == 0) {
                    const size_t o = ((size_t)u * L + (l - 1)) * nc;
#pragma unroll
                    for (int j = 0; j < GPL; ++j) {
                        const int col = j * 32 + lane;
                        if (col < nc) {
                            s.gs[q * np + col] = a.gall[o + col];
                            if (l < L) s.cs[q * np + col] = a.csall[o + col];
                        }
                    }
                }
            }
            for (int l = l0 + 1; !a.gall && l <= l1; ++l) {  // recompute g'^(l-1), cs^(l)
                const int q = l - l0 - 1;
                if (warp == 0) {
#pragma unroll
                    for (int j = 0; j < GPL; ++j)
                        if (j * 32 + lane < nc) s.gs[q * np + j * 32 + lane] = gm[j];
                }
                if (l == L) break;  // the output layer needs g'^(L-1) only
                fwd_iter<NCB, R, EXACT>(s, ld, nc, i0, vr, sc, gm, csum, par, lane, warp, W);
                if (warp == 0) {
#pragma unroll
                    for (int j = 0; j < GPL; ++j)
                        if (j * 32 + lane < nc) s.cs[q * np + j * 32 + lane] = csum[j];
                }
            }
            __syncthreads();  // the segment's g'^(l-1) and cs^(l) visible
            for (int l = l1; l > l0; --l) {
                const int q = l - l0 - 1;
                float gq[GPL], gcm[GPL];
#pragma unroll
                for (int j = 0; j < GPL; ++j) {
                    const int col = j * 32 + lane;
                    gq[j] = col < nc ? s.gs[q * np + col] : 0.f;
                    gcm[j] = (l < L && col < nc) ? gb[j] / fmaxf(s.cs[q * np + col], 1e-37f) : 0.f;
                }
                float gk[NCB], gck[NCB], acc[NCB];
                bcast_g<NCB, GPL>(gq, gk);
                bcast_g<NCB, GPL>(gcm, gck);
#pragma unroll
                for (int k = 0; k < NCB; ++k) acc[k] = 0.f;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (!vr[r]) continue;
                    const int i = i0 + r;
                    float p[NCB];
                    row_policy<NCB, EXACT>(s.C, ld, i, nc, sc, gk, p);
                    if (l == L) {  // output layer: p is the emitted policy x
                        const float wr = __ldg(a.omega + i) * s.r[i];  // dL/dx_ik = wr e_k
                        float h = 0.f, v = 0.f;
#pragma unroll
                        for (int k = 0; k < NCB; ++k) {
                            h += p[k] * (wr * s.e[k]);
                            if (k < a.K) v += s.e[k] * p[k];
                        }
                        vi[r] = v;
#pragma unroll
                        for (int k = 0; k < NCB; ++k) {
                            const float z = inv_eps * p[k] * (wr * s.e[k] - h);
                            dc[r][k] -= z;
                            acc[k] += z;
                        }
                    } else {
                        float ai = 0.f;
#pragma unroll
                        for (int k = 0; k < NCB; ++k) ai += p[k] * gck[k];
#pragma unroll
                        for (int k = 0; k < NCB; ++k) {
                            dc[r][k] += p[k] * (gck[k] - ai);
                            acc[k] += p[k] * ai;
                        }
                    }
                }
                if (l > 1) {  // gbar^(l-1); the warm start g^(0) is a constant
                    p2::column_sum<NCB, GPL>(acc, gb, nc, s.red, par, lane, warp, W);
                    par ^= 1;
                }
            }
            __syncthreads();  // the next segment rewrites gs / cs
        }

        if constexpr (MODE == ADJ_GRAD) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (!vr[r]) continue;
                const int i = i0 + r;
#pragma unroll
                for (int k = 0; k < NCB; ++k)
                    if (EXACT || k < nc) a.dC[((size_t)u * I + i) * nc + k] = dc[r][k];
                if (a.dr) a.dr[(size_t)u * I + i] = __ldg(a.omega + i) * vi[r];
            }
        } else {
            // optimiser step on the consumer's costs (ascent; Adam as in the fused step kernel)
#pragma unroll
            for (int k = 0; k < NCB; ++k) {
                if (!EXACT && k >= nc) break;
                if (i0 >= ld) break;
                const size_t off = ((size_t)u * nc + k) * ld + i0;
                float cv[R], mm[R], vv[R];
                ldv<R>(cv, s.C + k * ld + i0);
                if (a.optimizer == 0) {
                    ldv<R>(mm, a.m1 + off);
                    ldv<R>(vv, a.m2 + off);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    if (!vr[r]) continue;
                    const float g = dc[r][k];
                    gn2 += (double)(g * g);
                    if (a.optimizer == 1) {
                        cv[r] += a.lr * g;
                    } else {
                        mm[r] = a.beta1 * mm[r] + (1.f - a.beta1) * g;
                        vv[r] = a.beta2 * vv[r] + (1.f - a.beta2) * g * g;
                        const float sq = vv[r] > 0.f ? vv[r] * rsqrtf(vv[r]) : 0.f;
                        cv[r] += __fdividef(step_size * mm[r], fmaf(sq, inv_bc2s, a.adam_eps));
                    }
                }
                stv<R>(a.C + off, cv);
                if (a.optimizer == 0) {
                    stv<R>(a.m1 + off, mm);
                    stv<R>(a.m2 + off, vv);
                }
            }
        }
        __syncthreads();  // every read of the staged tile is done: stage the next consumer
        if (tid == 0) stage(a, u + gridDim.x, nc, ld, s);
    }

    if constexpr (MODE == ADJ_STEP) {  // CTA sum of the squared gradient, fixed order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gn2 += __shfl_xor_sync(FULL, gn2, o);
        if (lane == 0) s.dred[warp] = gn2;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < W; ++w) t += s.dred[w];
            a.gn2_part[blockIdx.x] = t;
        }
    }
}

}  // namespace p1adj
}  // namespace fr
