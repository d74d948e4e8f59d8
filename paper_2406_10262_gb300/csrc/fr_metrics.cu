// fr_metrics.cu -- the evaluation metrics of Sec. 4.1 on the GPU (fr_metrics).
//
//   v_uj      = sum_{k<K} e_k x_ujk                       one pass over the policy (value kernels)
//   E_ij      = sum_u r(u,i) v_uj = Imp_i(X_j)            dense |I| x |I| contraction over consumers
//   envy_i    = max_j E_ij - E_ii  (j = i allowed)        fused into the contraction's epilogue
//   Imp^unif_i = (sum_u r(u,i)) (sum_{k<K} e_k) / |I|     the uniform policy x_uik = b_k / |I|
//   better / worse: Imp_i > 1.1 Imp^unif_i / Imp_i < 0.9 Imp^unif_i (strict)
//
// The contraction runs on the tensor cores (fr_envy_tc.cu); its epilogue keeps only the row maxima
// of each tile and, on diagonal tiles, E_ii: the |I|^2 matrix is never written.
#include <cuda_bf16.h>

#include "fr_device.cuh"
#include "fr_internal.h"

namespace fr {

namespace {

__device__ __forceinline__ float rval(const void* r, int bf16, size_t o) {
    return bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(r)[o])
                : static_cast<const float*>(r)[o];
}

// v of consumer blockIdx.x under the free-cost policy (same arithmetic as policy_kernel). The
// column constants are staged in shared memory once per consumer; the row maximum takes one pass
// without exponentials and the normalisation a reciprocal.
__global__ void v_p1_kernel(const P1Args a, float* __restrict__ V) {
    __shared__ float s_gp[64], s_e[64];
    const int u = blockIdx.x;
    const int nc = a.nc;
    const float* C = a.C + (size_t)u * nc * a.ld;
    for (int k = threadIdx.x; k < nc; k += blockDim.x) {
        s_gp[k] = a.gP[(size_t)u * nc + k];
        s_e[k] = k < a.K ? a.e[k] : 0.f;
    }
    __syncthreads();
    const float sc = a.inv_eps_ln2;
    for (int i = threadIdx.x; i < a.ld; i += blockDim.x) {
        float v = 0.f;
        if (i < a.I) {
            float M = -INFINITY;
            for (int k = 0; k < nc; ++k) M = fmaxf(M, fmaf(-C[(size_t)k * a.ld + i], sc, s_gp[k]));
            float S = 0.f, num = 0.f;
            for (int k = 0; k < nc; ++k) {
                const float p = ex2(fmaf(-C[(size_t)k * a.ld + i], sc, s_gp[k]) - M);
                S += p;
                num = fmaf(s_e[k], p, num);
            }
            v = num * rcp_approx(S);
        }
        V[(size_t)u * a.ld + i] = v;
    }
}

// v under the per-item policy x_ik = softmax_k(g'_k + s_i (e_k - e_max)): the consumer's column
// constants are held in registers for a compiled column bucket NCB >= nc (the padding columns get
// g' = -inf, so their terms vanish), the row maximum takes one pass without exponentials and the
// normalisation a reciprocal.
template <int NCB>
__global__ void v_p2_kernel(const P2Args a, float* __restrict__ V) {
    const int u = blockIdx.x;
    const int nc = a.nc;
    float gk[NCB], ehk[NCB], ek[NCB];
#pragma unroll
    for (int k = 0; k < NCB; ++k) {
        gk[k] = k < nc ? __ldg(a.gP + (size_t)u * nc + k) : -INFINITY;
        ehk[k] = k < nc ? __ldg(a.e + k) - a.emax : 0.f;
        ek[k] = k < a.K ? __ldg(a.e + k) : 0.f;
    }
    for (int i = threadIdx.x; i < a.ld; i += blockDim.x) {
        float v = 0.f;
        if (i < a.I) {
            const float si = rval(a.r, a.r_bf16, (size_t)u * a.ld + i) * __ldg(a.w + i) * a.inv_eps_ln2;
            float M = -INFINITY;
#pragma unroll
            for (int k = 0; k < NCB; ++k) M = fmaxf(M, fmaf(si, ehk[k], gk[k]));
            float S = 0.f, num = 0.f;
#pragma unroll
            for (int k = 0; k < NCB; ++k) {
                const float p = ex2(fmaf(si, ehk[k], gk[k]) - M);
                S += p;
                num = fmaf(ek[k], p, num);
            }
            v = num * rcp_approx(S);
        }
        V[(size_t)u * a.ld + i] = v;
    }
}

// sum_u r(u,i): chunk blockIdx.y of COLSUM_CHUNKS interleaved consumer chunks, one thread per item
// (coalesced across items), compensated FP32 sums (Knuth's TwoSum) written as FP64 partials
// part[chunk][i]; colsum_final_kernel adds the chunks in a fixed order.
constexpr int COLSUM_CHUNKS = 32;

__global__ void colsum_kernel(const void* __restrict__ r, int r_bf16, int U, int I, int ld,
                              double* __restrict__ part) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I) return;
    float s = 0.f, c = 0.f;
    for (int u = blockIdx.y; u < U; u += COLSUM_CHUNKS) {
        const float x = rval(r, r_bf16, (size_t)u * ld + i);
        const float t = __fadd_rn(s, x);
        const float bp = __fsub_rn(t, s);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
        s = t;
    }
    part[(size_t)blockIdx.y * ld + i] = (double)s + (double)c;
}

__global__ void colsum_final_kernel(const double* __restrict__ part, int I, int ld,
                                    double* __restrict__ ru) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I) return;
    double s = 0.0;
    for (int q = 0; q < COLSUM_CHUNKS; ++q) s += part[(size_t)q * ld + i];
    ru[i] = s;
}

// envy_i = max over column tiles - E_ii; sum in FP64 (one CTA, fixed order). Uniform-policy
// impacts from the column sums of r and the strict 10% ratio tests against Imp_i.
__global__ void __launch_bounds__(1024) envy_final_kernel(const float* __restrict__ rmax, int ntj,
                                                          const float* __restrict__ diag,
                                                          const double* __restrict__ ru, int I,
                                                          int ld, const double* __restrict__ imp,
                                                          double esum, double* __restrict__ out,
                                                          double* __restrict__ env_item) {
    __shared__ double s_env[32];
    __shared__ int s_cnt[2][32];
    double env = 0.0;
    int nb = 0, nw = 0;
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        float m = -INFINITY;
        for (int t = 0; t < ntj; ++t) m = fmaxf(m, rmax[(size_t)t * ld + i]);
        const double env_i = (double)m - (double)diag[i];
        env += env_i;
        if (env_item) env_item[i] = env_i;
        const double unif = ru[i] * esum / I;
        if (imp[i] > 1.1 * unif) ++nb;
        if (imp[i] < 0.9 * unif) ++nw;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        env += __shfl_xor_sync(FULL, env, o);
        nb += __shfl_xor_sync(FULL, nb, o);
        nw += __shfl_xor_sync(FULL, nw, o);
    }
    if (lane == 0) {
        s_env[warp] = env;
        s_cnt[0][warp] = nb;
        s_cnt[1][warp] = nw;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double e = 0.0;
        int b = 0, w = 0;
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) {
            e += s_env[j];
            b += s_cnt[0][j];
            w += s_cnt[1][j];
        }
        out[0] = e / I;
        out[1] = 100.0 * b / I;
        out[2] = 100.0 * w / I;
    }
}

}  // namespace

cudaError_t launch_v_p1(const P1Args& a, float* V, cudaStream_t s) {
    v_p1_kernel<<<a.U, 256, 0, s>>>(a, V);
    return cudaGetLastError();
}

cudaError_t launch_v_p2(const P2Args& a, float* V, cudaStream_t s) {
    switch (a.nc) {  // exact column counts of the common shapes (K = 5, 10, 20), buckets otherwise
        case 6: v_p2_kernel<6><<<a.U, 256, 0, s>>>(a, V); break;
        case 11: v_p2_kernel<11><<<a.U, 256, 0, s>>>(a, V); break;
        case 21: v_p2_kernel<21><<<a.U, 256, 0, s>>>(a, V); break;
        default:
            if (a.nc <= 8)
                v_p2_kernel<8><<<a.U, 256, 0, s>>>(a, V);
            else if (a.nc <= 16)
                v_p2_kernel<16><<<a.U, 256, 0, s>>>(a, V);
            else
                v_p2_kernel<32><<<a.U, 256, 0, s>>>(a, V);
    }
    return cudaGetLastError();
}

int colsum_chunks() { return COLSUM_CHUNKS; }

cudaError_t launch_envy(const void* r, int r_bf16, const float* V, int U, int I, int ld,
                        const double* imp, double esum, float* rmax, float* diag, double* ru,
                        double* ru_part, double* out, double* env_item, int* err,
                        unsigned max_polls, void* planes, cudaStream_t s) {
    const int nt = envy_tc_col_tiles(I);  // rows of rmax written by the contraction
    cudaError_t e = launch_envy_tc(r, r_bf16, V, U, I, ld, rmax, diag, err, max_polls, planes, s);
    if (e != cudaSuccess) return e;
    colsum_kernel<<<dim3((I + 255) / 256, COLSUM_CHUNKS), 256, 0, s>>>(r, r_bf16, U, I, ld, ru_part);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    colsum_final_kernel<<<(I + 255) / 256, 256, 0, s>>>(ru_part, I, ld, ru);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    envy_final_kernel<<<1, 1024, 0, s>>>(rmax, nt, diag, ru, I, ld, imp, esum, out, env_item);
    return cudaGetLastError();
}


// ---- Frank-Wolfe certificate -------------------------------------------------------------------
// F is concave in X and every X_u lies in the transportation polytope of Eqs. (1)-(3), so
//   F* - F(X) <= max_Y <grad F(X), Y - X>,  dF/dx_uik = r(u,i) e_k / Imp_i  (e_k = 0 for the dummy).
// With e non-increasing the maximising Y_u puts the K items with the largest rho_ui = r(u,i)/Imp_i
// into slots 1..K in that order (rearrangement inequality), so per consumer
//   gap_u = sum_{k<K} e_k rho_u(k) - sum_i rho_ui sum_{k<K} e_k x_uik,
// and gap = sum_u gap_u >= F* - F(X) for exactly feasible X. The emitted X has exact rows and a
// small column residual, reported beside it: max_{u,k} |sum_i x_uik - b_k|.
namespace {

template <int MAXM>
__global__ void __launch_bounds__(256) cert_kernel(const P1Args a1, const P2Args a2, int p2,
                                                   const double* __restrict__ imp,
                                                   double* __restrict__ gap_part,
                                                   float* __restrict__ res_part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int U = p2 ? a2.U : a1.U, I = p2 ? a2.I : a1.I, K = p2 ? a2.K : a1.K;
    const int nc = p2 ? a2.nc : a1.nc, ld = p2 ? a2.ld : a1.ld;
    const float* e = p2 ? a2.e : a1.e;
    double* rho = reinterpret_cast<double*>(smem_raw);             // [I]
    float* csw = reinterpret_cast<float*>(rho + I);                 // [W][MAXM]
    __shared__ double s_red[32];
    __shared__ int s_idx[32];
    __shared__ float s_resm;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    double gap_acc = 0.0;
    float res_max = 0.f;
    for (int u = blockIdx.x; u < U; u += gridDim.x) {
        const float* gp = (p2 ? a2.gP : a1.gP) + (size_t)u * nc;
        float cs[MAXM];
#pragma unroll
        for (int k = 0; k < MAXM; ++k) cs[k] = 0.f;
        double lin = 0.0;
        for (int i = tid; i < I; i += blockDim.x) {
            float z[MAXM];
            float M = -INFINITY;
            float si = 0.f;
            if (p2) {
                const float ri = p2 ? (a2.r_bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(a2.r)[(size_t)u * ld + i])
                                                 : static_cast<const float*>(a2.r)[(size_t)u * ld + i])
                                    : 0.f;
                si = ri * a2.w[i] * a2.inv_eps_ln2;
            }
#pragma unroll
            for (int k = 0; k < MAXM; ++k) {
                if (k < nc) {
                    z[k] = p2 ? fmaf(si, e[k] - a2.emax, gp[k])
                              : gp[k] - a1.C[((size_t)u * nc + k) * ld + i] * a1.inv_eps_ln2;
                    M = fmaxf(M, z[k]);
                } else {
                    z[k] = -INFINITY;
                }
            }
            float S = 0.f;
#pragma unroll
            for (int k = 0; k < MAXM; ++k) {
                z[k] = k < nc ? ex2(z[k] - M) : 0.f;
                S += z[k];
            }
            const float inv = 1.f / S;
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < MAXM; ++k) {
                const float x = z[k] * inv;
                cs[k] += x;
                if (k < K) v += (double)e[k] * x;
            }
            const float r = p2 ? (a2.r_bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(a2.r)[(size_t)u * ld + i])
                                            : static_cast<const float*>(a2.r)[(size_t)u * ld + i])
                               : a1.r[(size_t)u * ld + i];
            const double rh = (double)r / imp[i];
            rho[i] = rh;
            lin += rh * v;
        }
        // column sums: warp shuffles, then per-warp partials in shared memory (fixed order)
#pragma unroll
        for (int k = 0; k < MAXM; ++k) {
            float c = cs[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(FULL, c, o);
            if (lane == 0) csw[warp * MAXM + k] = c;
        }
        // lin: block sum in fixed order
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lin += __shfl_xor_sync(FULL, lin, o);
        if (lane == 0) s_red[warp] = lin;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < W; ++w) t += s_red[w];
            gap_acc -= t;
            float rm = 0.f;
            for (int k = 0; k < nc; ++k) {
                float c = 0.f;
                for (int w = 0; w < W; ++w) c += csw[w * MAXM + k];
                const float bk = k < K ? 1.f : (float)(I - K);  // Eq. (2) and the dummy mass
                rm = fmaxf(rm, fabsf(c - bk));
            }
            s_resm = rm;
        }
        __syncthreads();
        if (tid == 0) res_max = fmaxf(res_max, s_resm);
        // top-K of rho by K rounds of a CTA-wide arg-max (taken entries become -inf)
        for (int k = 0; k < K; ++k) {
            double best = -INFINITY;
            int bi = -1;
            for (int i = tid; i < I; i += blockDim.x)
                if (rho[i] > best) { best = rho[i]; bi = i; }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(FULL, best, o);
                const int oi = __shfl_xor_sync(FULL, bi, o);
                if (ob > best || (ob == best && oi >= 0 && (bi < 0 || oi < bi))) { best = ob; bi = oi; }
            }
            if (lane == 0) { s_red[warp] = best; s_idx[warp] = bi; }
            __syncthreads();
            if (tid == 0) {
                double bb = -INFINITY;
                int ii = -1;
                for (int w = 0; w < W; ++w)
                    if (s_red[w] > bb || (s_red[w] == bb && s_idx[w] >= 0 && (ii < 0 || s_idx[w] < ii))) {
                        bb = s_red[w];
                        ii = s_idx[w];
                    }
                if (ii >= 0) {
                    gap_acc += (double)e[k] * bb;
                    rho[ii] = -INFINITY;
                }
            }
            __syncthreads();
        }
    }
    if (tid == 0) {
        gap_part[blockIdx.x] = gap_acc;
        res_part[blockIdx.x] = res_max;
    }
}

__global__ void cert_final_kernel(const double* __restrict__ gap_part,
                                  const float* __restrict__ res_part, int G, double* out) {
    if (threadIdx.x != 0) return;
    double g = 0.0;
    float r = 0.f;
    for (int j = 0; j < G; ++j) {
        g += gap_part[j];
        r = fmaxf(r, res_part[j]);
    }
    out[0] = g;
    out[1] = (double)r;
}

}  // namespace

int cert_grid(int U, int sms) { return U < 4 * sms ? U : 4 * sms; }

size_t cert_smem(int I) { return sizeof(double) * (size_t)I + sizeof(float) * 8 * 64; }

cudaError_t launch_certificate(const P1Args* a1, const P2Args* a2, const double* imp, int nc, int I,
                               int G, double* gap_part, float* res_part, double* out, cudaStream_t s) {
    const P1Args z1{};
    const P2Args z2{};
    const P1Args& p1 = a1 ? *a1 : z1;
    const P2Args& q2 = a2 ? *a2 : z2;
    const int p2 = a2 != nullptr;
    const size_t sm = cert_smem(I);
    cudaError_t e;
    if (nc <= 16) {
        if ((e = raise_smem_limit((const void*)cert_kernel<16>, sm)) != cudaSuccess) return e;
        cert_kernel<16><<<G, 256, sm, s>>>(p1, q2, p2, imp, gap_part, res_part);
    } else if (nc <= 32) {
        if ((e = raise_smem_limit((const void*)cert_kernel<32>, sm)) != cudaSuccess) return e;
        cert_kernel<32><<<G, 256, sm, s>>>(p1, q2, p2, imp, gap_part, res_part);
    } else {
        if ((e = raise_smem_limit((const void*)cert_kernel<64>, sm)) != cudaSuccess) return e;
        cert_kernel<64><<<G, 256, sm, s>>>(p1, q2, p2, imp, gap_part, res_part);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cert_final_kernel<<<1, 32, 0, s>>>(gap_part, res_part, G, out);
    return cudaGetLastError();
}

}  // namespace fr
