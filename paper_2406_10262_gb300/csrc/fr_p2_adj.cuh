// fr_p2_adj.cuh -- unrolled gradient of the per-item parametrisation: the adjoint of the L Sinkhorn
// iterations of Problem (7) (Sec. 3), in reverse, with the column potentials checkpointed.
//
// Forward map of one consumer (natural units, iteration l = 1..L, as the sweep runs it):
//   P^(l)_ik = softmax_k((g^(l-1)_k - c_ik) / eps)                 row update (Eq. 1)
//   g^(l)_k  = g^(l-1)_k + eps (log b_k - log cs^(l)_k),  cs^(l)_k = sum_i P^(l)_ik   (Eq. 2)
//   x = P^(L)                                                       the emitted policy
// Reverse sweep for L = sum_i omega_i Imp_i, dL/dx_ik = omega_i r_i e_k =: gx_ik (e of the dummy = 0):
//   output layer: zbar_ik = x_ik (gx_ik - h_i), h_i = sum_k x_ik gx_ik,
//                 dc_ik -= zbar_ik / eps,  gbar^(L-1)_k = sum_i zbar_ik / eps
//   l = L-1 .. 1: gc_k = gbar^(l)_k / cs^(l)_k,  a_i = sum_k P^(l)_ik gc_k,
//                 dc_ik += P^(l)_ik (gc_k - a_i),  gbar^(l-1)_k = sum_i P^(l)_ik a_i
// (through the column update g^(l) depends on f^(l) with weight -P/cs and on c with +P/cs; through
// the row update f^(l) depends on g^(l-1) with weight -P and on c with +P). g^(0) is the warm start,
// a constant. Only rho_i = sum_k e_k dc_ik is kept, since dc_ik/dtheta_i = -r_i e_k w_i:
//   dL/dtheta_i += -r_i w_i rho_i,   dL/dr(u,i) = omega_i v_i - w_i rho_i,  v_i = sum_{k<K} e_k x_ik.
// Because sum_k P_ik (gc_k - a_i) = 0, e_k may be replaced by e_k - e_max in the rho terms of the
// reverse iterations, which keeps every sum in the packed registers of the sweep. The output layer's
// term is a variance, sum_k e_k zbar_ik = omega_i r_i sum_k x_ik (e_k - ebar_i)^2 with ebar_i =
// sum_k x_ik e_k; it is summed in that centred form: the uncentred form sum_k e_k x_ik (e_k - ebar_i)
// cancels catastrophically for rows whose policy is nearly deterministic, turning the FP32 rounding
// of the row normaliser into errors of ~1e-5 relative in dL/dtheta.
//
// Checkpointing: the sweep stores g^(j ce) for j = 0 .. ceil(L/ce)-1. Segment j (iterations
// j ce + 1 .. min((j+1) ce, L)) is recomputed from its checkpoint with the same arithmetic as the
// sweep, keeping g^(l-1) and cs^(l) of the segment in shared memory (2 ce m floats), then reversed.
// Work: L forward plus L reverse iterations per consumer; memory: ceil(L/ce) m floats per consumer.
// With a checkpoint every iteration (ce = 1) the sweep also keeps each iteration's column sums
// (P2Args::csk, L m more floats per consumer), and the re-runs reduce to loading them: L reverse
// iterations per consumer.
#pragma once
#include "fr_p2.cuh"

namespace fr {
namespace p2 {

struct AdjSmem {
    float* acc;   // [ld] per-CTA dL/dtheta partials
    float* drt;   // [ld] omega_i v_i of the current consumer
    unsigned char* rbuf;  // [2][ld] staged relevance rows
    float* e;     // [ncx]
    float* eh;    // [ncx] e_k - e_max (0 beyond nc)
    float* ib;    // [ncx] 1 / b_k
    float* gs;    // [ce][ncp] g^(l-1) of the segment
    float* cs;    // [ce][ncp] cs^(l) of the segment
    float* red;   // [2 * W * P]
    unsigned long long* bar;  // [2]
};

__host__ __device__ inline size_t adj_layout(int ncb, int nc, int ld, int W, int esz, int ce,
                                             AdjSmem* s, unsigned char* base) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 15) / 16 * 16;
        return o;
    };
    const int P = pow2ceil(ncb), nx = ncx(nc, ncb), np = ncp(nc);
    const size_t o_bar = take(2 * sizeof(unsigned long long));
    const size_t o_acc = take(sizeof(float) * ld), o_drt = take(sizeof(float) * ld);
    const size_t o_rb = take((size_t)2 * esz * ld);
    const size_t o_e = take(sizeof(float) * nx), o_eh = take(sizeof(float) * nx);
    const size_t o_ib = take(sizeof(float) * nx);
    const size_t o_gs = take(sizeof(float) * (size_t)ce * np);
    const size_t o_cs = take(sizeof(float) * (size_t)ce * np);
    const size_t o_red = take(sizeof(float) * 2 * W * P);
    if (s) {
        s->bar = (unsigned long long*)(base + o_bar);
        s->acc = (float*)(base + o_acc);
        s->drt = (float*)(base + o_drt);
        s->rbuf = base + o_rb;
        s->e = (float*)(base + o_e);
        s->eh = (float*)(base + o_eh);
        s->ib = (float*)(base + o_ib);
        s->gs = (float*)(base + o_gs);
        s->cs = (float*)(base + o_cs);
        s->red = (float*)(base + o_red);
    }
    return off;
}

// Loads lane-distributed potentials into per-thread registers: gk (all columns, -inf padding
// unless EXACT), packed pairs g2 and the unpaired last column gt.
template <int NCB, int GPL, bool EXACT>
__device__ __forceinline__ void adj_bcast(const float (&gm)[GPL], int nc, float (&gk)[NCB],
                                          f2* g2, float& gt) {
    bcast_g<NCB, GPL>(gm, gk);
    if (!EXACT) {
#pragma unroll
        for (int k = 0; k < NCB; ++k)
            if (k >= nc) gk[k] = -INFINITY;
    }
#pragma unroll
    for (int j = 0; j < NCB / 2; ++j) g2[j] = pk(gk[2 * j], gk[2 * j + 1]);
    gt = NCB % 2 == 1 ? gk[NCB - 1] : 0.f;
}

// Two CTAs of 256 threads per SM (at most 128 registers) where the live set fits without spills
// (8 rows per thread, up to 21 columns); one otherwise.
template <int NCB, int R>
constexpr int adj_min_blocks() { return (R <= 8 && NCB <= 21) ? 2 : 1; }

template <int NCB, int R, bool EXACT>
__global__ void __launch_bounds__(256, adj_min_blocks<NCB, R>()) p2_adj_kernel(const P2Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int GPL = (NCB + 31) / 32;
    constexpr int NP = NCB / 2;
    constexpr int NPA = NP > 0 ? NP : 1;
    constexpr bool TAIL = NCB % 2 == 1;
    const int nc = EXACT ? NCB : a.nc;
    const int nx = ncx(nc, NCB), np_ = ncp(nc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int T = blockDim.x;
    const int I = a.I, ld = a.ld, L = a.L, ce = a.ce;
    const int i0 = tid * R;
    const bool bf16 = a.r_bf16 != 0;
    const int esz = bf16 ? 2 : 4;
    const float inv_eps = a.inv_eps;
    AdjSmem s;
    adj_layout(NCB, nc, ld, W, esz, ce, &s, smem_raw);

    if (a.st->stop) return;

    if (tid == 0) {
        mbar_init(s.bar, 1);
        mbar_init(s.bar + 1, 1);
        fence_mbar_init();
    }
    __syncthreads();  // mbarriers initialised before any wait
    if (tid == 0) p2_stage(a, blockIdx.x, 0, s.bar, s.rbuf, esz);
    for (int i = tid; i < ld; i += T) s.acc[i] = 0.f;
    for (int k = tid; k < nx; k += T) {
        s.e[k] = k < nc ? a.e[k] : 0.f;
        s.eh[k] = k < nc ? a.e[k] - a.emax : 0.f;
        s.ib[k] = k < nc ? a.invb[k] : 0.f;
    }
    __syncthreads();
    f2 e2[NPA];
#pragma unroll
    for (int j = 0; j < NP; ++j) e2[j] = pk(s.eh[2 * j], s.eh[2 * j + 1]);
    const float et = TAIL ? s.eh[NCB - 1] : 0.f;
    const int ref = nc - 1;
    bool vr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) vr[r] = i0 + r < I;

    int par = 0;
    unsigned phase_bits = 0u;
    int b = 0;
    for (int u = blockIdx.x; u < a.U; u += gridDim.x, b ^= 1) {
        // the consumer's relevance row is the only copy in flight; if the bounded wait expires,
        // the CTA records a timeout, waits (default bound) for the copy to land and stops
        const bool row_ok = cta_wait_or_drain(s.bar + b, (phase_bits >> b) & 1u, a.max_polls,
                                              kDefaultPolls, &a.st->err, 4);
        phase_bits ^= 1u << b;
        if (!row_ok) break;
        const unsigned char* rrow = s.rbuf + (size_t)b * esz * ld;
        float sv[R], rho[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            sv[r] = vr[r] ? load_r(rrow, i0 + r, bf16) * __ldg(a.w + i0 + r) * a.inv_eps_ln2 : 0.f;
            rho[r] = 0.f;
        }
        float gb[GPL];  // adjoint of the column potentials (natural units), lane-distributed
#pragma unroll
        for (int j = 0; j < GPL; ++j) gb[j] = 0.f;

        for (int seg = a.nck - 1; seg >= 0; --seg) {
            const int l0 = seg * ce;
            const int l1 = min(l0 + ce, L);
            // ---- recompute the segment from its checkpoint g^(l0)
            float gm[GPL];
#pragma unroll
            for (int j = 0; j < GPL; ++j) {
                const int col = j * 32 + lane;
                gm[j] = col < nc ? a.ck[((size_t)u * a.nck + seg) * nc + col] : 0.f;
            }
            for (int l = l0 + 1; l <= l1; ++l) {
                const int q = l - l0 - 1;
                if (warp == 0) {
#pragma unroll
                    for (int j = 0; j < GPL; ++j)
                        if (j * 32 + lane < nc) s.gs[q * np_ + j * 32 + lane] = gm[j];
                }
                if (l == L) break;  // the output layer needs g^(L-1) only
                float csum[GPL];
                if (a.csk) {  // the sweep kept this iteration's column sums: no row work
#pragma unroll
                    for (int j = 0; j < GPL; ++j) {
                        const int col = j * 32 + lane;
                        csum[j] = col < nc ? a.csk[((size_t)u * L + (l - 1)) * nc + col] : 0.f;
                    }
                } else {
                    float gk[NCB];
                    f2 g2[NPA];
                    float gt;
                    adj_bcast<NCB, GPL, EXACT>(gm, nc, gk, g2, gt);
                    f2 cs2[NPA];
#pragma unroll
                    for (int j = 0; j < NP; ++j) cs2[j] = 0ull;
                    float cst = 0.f;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (!vr[r]) continue;
                        f2 p2[NPA];
                        float pt;
                        const float inv = p2_row<NCB, EXACT>(sv[r], e2, et, g2, gt, s.eh, gk, nc, p2, pt);
                        const f2 inv2 = pk(inv, inv);
#pragma unroll
                        for (int j = 0; j < NP; ++j) cs2[j] = fma2(p2[j], inv2, cs2[j]);
                        cst = fmaf(pt, inv, cst);
                    }
                    float csv[NCB];
#pragma unroll
                    for (int j = 0; j < NP; ++j) upk(cs2[j], csv[2 * j], csv[2 * j + 1]);
                    if (TAIL) csv[NCB - 1] = cst;
                    column_sum<NCB, GPL>(csv, csum, nc, s.red, par, lane, warp, W);
                    par ^= 1;
                }
#pragma unroll
                for (int j = 0; j < GPL; ++j) {
                    const int col = j * 32 + lane;
                    if (col < nc) {
                        gm[j] -= log2_near1(fmaxf(csum[j] * s.ib[col], 1e-37f));  // as the sweep
                        if (warp == 0) s.cs[q * np_ + col] = csum[j];
                    }
                }
                const float gref = __shfl_sync(FULL, gm[ref / 32], ref % 32);
#pragma unroll
                for (int j = 0; j < GPL; ++j) gm[j] -= gref;
            }
            __syncthreads();  // gs / cs of the segment visible to every warp
            if (seg == a.nck - 1 && tid == 0) p2_stage(a, u + gridDim.x, b ^ 1, s.bar, s.rbuf, esz);

            // ---- reverse through iterations l1 .. l0 + 1
            for (int l = l1; l > l0; --l) {
                const int q = l - l0 - 1;
                float gmq[GPL], gcm[GPL];
#pragma unroll
                for (int j = 0; j < GPL; ++j) {
                    const int col = j * 32 + lane;
                    gmq[j] = col < nc ? s.gs[q * np_ + col] : 0.f;
                    gcm[j] = (l < L && col < nc) ? gb[j] / fmaxf(s.cs[q * np_ + col], 1e-37f) : 0.f;
                }
                float gk[NCB];
                f2 g2[NPA];
                float gt;
                adj_bcast<NCB, GPL, EXACT>(gmq, nc, gk, g2, gt);
                f2 acc2[NPA];
#pragma unroll
                for (int j = 0; j < NP; ++j) acc2[j] = 0ull;
                float acct = 0.f;
                if (l == L) {
                    // output layer: zbar_ik = x_ik omega_i r_i (eh_k - sum_k' x_ik' eh_k')
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (!vr[r]) continue;
                        f2 p2[NPA];
                        float pt;
                        const float inv = p2_row<NCB, EXACT>(sv[r], e2, et, g2, gt, s.eh, gk, nc, p2, pt);
                        f2 x2 = 0ull;
                        float v = 0.f;
#pragma unroll
                        for (int j = 0; j < NP; ++j) {
                            x2 = fma2(p2[j], e2[j], x2);
                            float p0, p1;
                            upk(p2[j], p0, p1);
                            if (2 * j < a.K) v += s.e[2 * j] * p0;
                            if (2 * j + 1 < a.K) v += s.e[2 * j + 1] * p1;
                        }
                        if (TAIL && NCB - 1 < a.K) v += s.e[NCB - 1] * pt;
                        float x0, x1;
                        upk(x2, x0, x1);
                        const float ehx = (x0 + x1 + (TAIL ? pt * et : 0.f)) * inv;
                        const int i = i0 + r;
                        const float om = __ldg(a.omega + i);
                        const float wr = om * load_r(rrow, i, bf16);
                        const float coef = inv_eps * wr * inv;
                        const f2 ehx2 = pk(ehx, ehx), coef2 = pk(coef, coef);
                        f2 rs2 = 0ull;
#pragma unroll
                        for (int j = 0; j < NP; ++j) {
                            const f2 dv = sub2(e2[j], ehx2);               // eh_k - ehx
                            const f2 y = fma2(p2[j], dv, 0ull);             // p_k (eh_k - ehx)
                            rs2 = fma2(dv, y, rs2);                         // centred variance
                            acc2[j] = fma2(coef2, y, acc2[j]);
                        }
                        float rs0, rs1;
                        upk(rs2, rs0, rs1);
                        float rs = rs0 + rs1;
                        if (TAIL) {
                            const float dv = et - ehx;
                            const float y = pt * dv;
                            rs = fmaf(dv, y, rs);
                            acct = fmaf(coef, y, acct);
                        }
                        rho[r] -= coef * rs;
                        s.drt[i] = om * (v * inv);
                    }
                } else {
                    // gc shifted by the gauge column's value c (the dummy's, which holds most of
                    // every row's mass): a_i - c stays small, and with d_k = eh_k (gc_k - c)
                    //   sum_k eh_k p_k (gc_k - a_i) = sum_k p_k d_k - (a_i - c) sum_k p_k eh_k
                    // takes three packed dot products per row instead of the centred form's five
                    // packed operations (the identity sum_k P_ik (gc_k - a_i) = 0 holds for any c)
                    float gck[NCB];
                    bcast_g<NCB, GPL>(gcm, gck);
                    const float gcc = __shfl_sync(FULL, gcm[ref / 32], ref % 32);
                    f2 gc2[NPA], d2[NPA];
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        gc2[j] = pk(gck[2 * j] - gcc, gck[2 * j + 1] - gcc);
                        d2[j] = mul2(e2[j], gc2[j]);
                    }
                    const float gct = TAIL ? gck[NCB - 1] - gcc : 0.f;
                    const float dt = et * gct;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (!vr[r]) continue;
                        f2 p2[NPA];
                        float pt;
                        const float inv = p2_row<NCB, EXACT>(sv[r], e2, et, g2, gt, s.eh, gk, nc, p2, pt);
                        f2 A2 = 0ull, B2 = 0ull, C2 = 0ull;
#pragma unroll
                        for (int j = 0; j < NP; ++j) {
                            A2 = fma2(p2[j], gc2[j], A2);
                            B2 = fma2(p2[j], d2[j], B2);
                            C2 = fma2(p2[j], e2[j], C2);
                        }
                        float A0, A1, B0, B1, C0, C1;
                        upk(A2, A0, A1);
                        upk(B2, B0, B1);
                        upk(C2, C0, C1);
                        float A = A0 + A1, B = B0 + B1, C = C0 + C1;
                        if (TAIL) {
                            A = fmaf(pt, gct, A);
                            B = fmaf(pt, dt, B);
                            C = fmaf(pt, et, C);
                        }
                        const float ai = A * inv;                 // a_i - c
                        rho[r] = fmaf(fmaf(-ai, C, B), inv, rho[r]);
                        const float iai = inv * (ai + gcc);       // P_ik a_i = p_ik iai
                        const f2 iai2 = pk(iai, iai);
#pragma unroll
                        for (int j = 0; j < NP; ++j) acc2[j] = fma2(p2[j], iai2, acc2[j]);
                        if (TAIL) acct = fmaf(pt, iai, acct);
                    }
                }
                if (l > 1) {  // gbar^(l-1); the warm start g^(0) is a constant
                    float csv[NCB];
#pragma unroll
                    for (int j = 0; j < NP; ++j) upk(acc2[j], csv[2 * j], csv[2 * j + 1]);
                    if (TAIL) csv[NCB - 1] = acct;
                    column_sum<NCB, GPL>(csv, gb, nc, s.red, par, lane, warp, W);
                    par ^= 1;
                }
            }
            __syncthreads();  // gs / cs are rewritten by the next segment
        }
        // dL/dtheta partials and dL/dr of this consumer
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (!vr[r]) continue;
            const int i = i0 + r;
            const float wi = __ldg(a.w + i);
            s.acc[i] -= load_r(rrow, i, bf16) * wi * rho[r];
            if (a.dr) a.dr[(size_t)u * I + i] = s.drt[i] - wi * rho[r];
        }
    }
    __syncthreads();
    for (int i = tid; i < ld; i += T) a.part[(size_t)blockIdx.x * ld + i] = s.acc[i];
}

template <int NCB, int R, bool EXACT>
void p2_make_adj(int threads, P2Variant* v) {
    v->adj = (const void*)p2_adj_kernel<NCB, R, EXACT>;
    v->adj_threads = threads;
}

}  // namespace p2
}  // namespace fr
