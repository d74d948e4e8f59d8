// fr_metrics.cu -- the evaluation metrics of Sec. 4.1 on the GPU (fr_metrics).
//
//   v_uj      = sum_{k<K} e_k x_ujk                       one pass over the policy (value kernels)
//   E_ij      = sum_u r(u,i) v_uj = Imp_i(X_j)            dense |I| x |I| contraction over consumers
//   envy_i    = max_j E_ij - E_ii  (j = i allowed)        fused into the contraction's epilogue
//   Imp^unif_i = (sum_u r(u,i)) (sum_{k<K} e_k) / |I|     the uniform policy x_uik = b_k / |I|
//   better / worse: Imp_i > 1.1 Imp^unif_i / Imp_i < 0.9 Imp^unif_i (strict)
//
// The contraction is an FP32 SIMT GEMM (E = R^T V, 64 x 64 tiles, 4 x 4 per thread, consumers
// streamed through shared memory 16 at a time) whose epilogue keeps only the row maxima of its
// tile and, on diagonal tiles, E_ii: the |I|^2 matrix is never written.
#include <cuda_bf16.h>

#include "fr_device.cuh"
#include "fr_internal.h"

namespace fr {

namespace {

constexpr int ET = 64;   // tile edge (items)
constexpr int EU = 16;   // consumers per shared-memory stage
constexpr int EMT = 4;   // micro tile edge per thread

__device__ __forceinline__ float rval(const void* r, int bf16, size_t o) {
    return bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(r)[o])
                : static_cast<const float*>(r)[o];
}

// v of consumers u0 + blockIdx.x under the free-cost policy (same arithmetic as policy_kernel).
__global__ void v_p1_kernel(const P1Args a, float* __restrict__ V) {
    const int u = blockIdx.x;
    const int nc = a.nc;
    const float* C = a.C + (size_t)u * nc * a.ld;
    const float* gp = a.gP + (size_t)u * nc;
    for (int i = threadIdx.x; i < a.ld; i += blockDim.x) {
        float v = 0.f;
        if (i < a.I) {
            float M = -INFINITY;
            for (int k = 0; k < nc; ++k) M = fmaxf(M, gp[k] - C[(size_t)k * a.ld + i] * a.inv_eps_ln2);
            float S = 0.f, num = 0.f;
            for (int k = 0; k < nc; ++k) {
                const float p = ex2(gp[k] - C[(size_t)k * a.ld + i] * a.inv_eps_ln2 - M);
                S += p;
                if (k < a.K) num += a.e[k] * p;
            }
            v = num / S;
        }
        V[(size_t)u * a.ld + i] = v;
    }
}

// v under the per-item policy x_ik = softmax_k(g'_k + s_i (e_k - e_max)).
__global__ void v_p2_kernel(const P2Args a, float* __restrict__ V) {
    const int u = blockIdx.x;
    const int nc = a.nc;
    const float* gp = a.gP + (size_t)u * nc;
    for (int i = threadIdx.x; i < a.ld; i += blockDim.x) {
        float v = 0.f;
        if (i < a.I) {
            const float si = rval(a.r, a.r_bf16, (size_t)u * a.ld + i) * a.w[i] * a.inv_eps_ln2;
            float M = -INFINITY;
            for (int k = 0; k < nc; ++k) M = fmaxf(M, fmaf(si, a.e[k] - a.emax, gp[k]));
            float S = 0.f, num = 0.f;
            for (int k = 0; k < nc; ++k) {
                const float p = ex2(fmaf(si, a.e[k] - a.emax, gp[k]) - M);
                S += p;
                if (k < a.K) num += a.e[k] * p;
            }
            v = num / S;
        }
        V[(size_t)u * a.ld + i] = v;
    }
}

// Tile (bi, bj) of E = R^T V: rows i in [64 bi, 64 bi + 64), columns j in [64 bj, ...). Writes the
// row maxima over the tile's valid columns to rmax[bj][i] and, on diagonal tiles, E_ii to diag[i].
__global__ void __launch_bounds__(256) envy_gemm_kernel(const void* __restrict__ r, int r_bf16,
                                                        const float* __restrict__ V, int U, int I,
                                                        int ld, float* __restrict__ rmax,
                                                        float* __restrict__ diag) {
    __shared__ __align__(16) float sr[EU][ET];
    __shared__ __align__(16) float sv[EU][ET];
    __shared__ float red[ET][ET / EMT + 1];
    const int tid = threadIdx.x;
    const int tx = tid % (ET / EMT), ty = tid / (ET / EMT);  // 16 x 16 threads
    const int i0 = blockIdx.y * ET, j0 = blockIdx.x * ET;
    float acc[EMT][EMT];
#pragma unroll
    for (int a = 0; a < EMT; ++a)
#pragma unroll
        for (int b = 0; b < EMT; ++b) acc[a][b] = 0.f;
    for (int u0 = 0; u0 < U; u0 += EU) {
        // 16 consumers x 64 items of r and of V; thread t loads 4 consecutive items of one row
        for (int q = tid; q < EU * ET / 4; q += blockDim.x) {
            const int uu = q / (ET / 4), c4 = (q % (ET / 4)) * 4;
            const int u = u0 + uu;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int ii = i0 + c4 + c, jj = j0 + c4 + c;
                sr[uu][c4 + c] = (u < U && ii < ld) ? rval(r, r_bf16, (size_t)u * ld + ii) : 0.f;
                sv[uu][c4 + c] = (u < U && jj < ld) ? V[(size_t)u * ld + jj] : 0.f;
            }
        }
        __syncthreads();
#pragma unroll
        for (int uu = 0; uu < EU; ++uu) {
            const float4 ra = *reinterpret_cast<const float4*>(&sr[uu][ty * EMT]);
            const float4 va = *reinterpret_cast<const float4*>(&sv[uu][tx * EMT]);
            const float rr[4] = {ra.x, ra.y, ra.z, ra.w}, vv[4] = {va.x, va.y, va.z, va.w};
#pragma unroll
            for (int a = 0; a < EMT; ++a)
#pragma unroll
                for (int b = 0; b < EMT; ++b) acc[a][b] = fmaf(rr[a], vv[b], acc[a][b]);
        }
        __syncthreads();
    }
    // epilogue: per-thread row maxima over its 4 columns, then over the 16 column groups
#pragma unroll
    for (int a = 0; a < EMT; ++a) {
        const int il = ty * EMT + a;
        float m = -INFINITY;
#pragma unroll
        for (int b = 0; b < EMT; ++b) {
            const int j = j0 + tx * EMT + b;
            if (j < I) m = fmaxf(m, acc[a][b]);
            if (blockIdx.x == blockIdx.y && j == i0 + il && j < I) diag[j] = acc[a][b];
        }
        red[il][tx] = m;
    }
    __syncthreads();
    if (tid < ET) {
        float m = -INFINITY;
        for (int t = 0; t < ET / EMT; ++t) m = fmaxf(m, red[tid][t]);
        const int i = i0 + tid;
        if (i < I) rmax[(size_t)blockIdx.x * ld + i] = m;
    }
}

// sum_u r(u,i) in FP64, one thread per item (coalesced across items).
__global__ void colsum_kernel(const void* __restrict__ r, int r_bf16, int U, int I, int ld,
                              double* __restrict__ ru) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= I) return;
    double s = 0.0;
    for (int u = 0; u < U; ++u) s += (double)rval(r, r_bf16, (size_t)u * ld + i);
    ru[i] = s;
}

// envy_i = max over column tiles - E_ii; sum in FP64 (one CTA, fixed order). Uniform-policy
// impacts from the column sums of r and the strict 10% ratio tests against Imp_i.
__global__ void __launch_bounds__(1024) envy_final_kernel(const float* __restrict__ rmax, int ntj,
                                                          const float* __restrict__ diag,
                                                          const double* __restrict__ ru, int I,
                                                          int ld, const double* __restrict__ imp,
                                                          double esum, double* __restrict__ out) {
    __shared__ double s_env[32];
    __shared__ int s_cnt[2][32];
    double env = 0.0;
    int nb = 0, nw = 0;
    for (int i = threadIdx.x; i < I; i += blockDim.x) {
        float m = -INFINITY;
        for (int t = 0; t < ntj; ++t) m = fmaxf(m, rmax[(size_t)t * ld + i]);
        env += (double)m - (double)diag[i];
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

int envy_tiles(int I) { return (I + ET - 1) / ET; }

cudaError_t launch_v_p1(const P1Args& a, float* V, cudaStream_t s) {
    v_p1_kernel<<<a.U, 256, 0, s>>>(a, V);
    return cudaGetLastError();
}

cudaError_t launch_v_p2(const P2Args& a, float* V, cudaStream_t s) {
    v_p2_kernel<<<a.U, 256, 0, s>>>(a, V);
    return cudaGetLastError();
}

cudaError_t launch_envy(const void* r, int r_bf16, const float* V, int U, int I, int ld,
                        const double* imp, double esum, float* rmax, float* diag, double* ru,
                        double* out, int* err, bool tensor_cores, cudaStream_t s) {
    int nt;
    cudaError_t e;
    if (tensor_cores) {
        nt = envy_tc_tiles(I);
        e = launch_envy_tc(r, r_bf16, V, U, I, ld, rmax, diag, err, s);
    } else {
        nt = envy_tiles(I);
        envy_gemm_kernel<<<dim3(nt, nt), 256, 0, s>>>(r, r_bf16, V, U, I, ld, rmax, diag);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    colsum_kernel<<<(I + 255) / 256, 256, 0, s>>>(r, r_bf16, U, I, ld, ru);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    envy_final_kernel<<<1, 1024, 0, s>>>(rmax, nt, diag, ru, I, ld, imp, esum, out);
    return cudaGetLastError();
}

}  // namespace fr
