// fr_p2_host.cu -- variant selection and launches of the per-item parametrisation, and the
// cross-consumer reduction of dL/dtheta with the optimiser step on theta.
#include <cuda_bf16.h>

#include "fr_device.cuh"
#include "fr_internal.h"
#include "fr_p2.cuh"

namespace fr {

namespace {

constexpr int AD_ITEMS = 32, AD_WARPS = 8;

// dL/dtheta_i = sum over the per-CTA partials (FP64, fixed order); its squared norm; the ascent
// step of Algorithm 1 on theta (Adam as in PyTorch with maximize=True, or SGD) and w = exp(theta).
// bid / nb: this CTA's index among the nb CTAs that update one problem.
__device__ __forceinline__ void adam_body(const P2AdamArgs& a, int bid, int nb) {
    __shared__ double s_sum[AD_WARPS][AD_ITEMS];
    __shared__ int s_last;
    if (a.st->stop) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int item = bid * AD_ITEMS + lane;
    double acc = 0.0;
    if (item < a.I)
        for (int g = warp; g < a.G; g += AD_WARPS) acc += (double)a.part[(size_t)g * a.ld + item];
    s_sum[warp][lane] = acc;
    __syncthreads();
    if (warp == 0) {
        double d = 0.0;
        for (int w = 0; w < AD_WARPS; ++w) d += s_sum[w][lane];
        double g2 = 0.0;
        if (item < a.I) {
            g2 = d * d;
            if (a.dtheta_out) a.dtheta_out[item] = (float)d;
            if (a.apply) {
                const float gr = (float)d;
                float th = a.theta[item];
                if (a.optimizer == 1) {
                    th += a.lr * gr;
                } else {
                    const float t1 = (float)(a.st->t + 1);
                    const float step = a.lr / one_minus_pow(a.beta1, t1);
                    const float bc2s = sqrtf(one_minus_pow(a.beta2, t1));
                    float m = a.m1[item], v = a.m2[item];
                    m = a.beta1 * m + (1.f - a.beta1) * gr;
                    v = a.beta2 * v + (1.f - a.beta2) * gr * gr;
                    th += step * m / (sqrtf(v) / bc2s + a.adam_eps);
                    a.m1[item] = m;
                    a.m2[item] = v;
                }
                a.theta[item] = th;
                a.w[item] = expf(th);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) g2 += __shfl_xor_sync(FULL, g2, o);
        if (lane == 0) a.blk[bid] = g2;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&a.st->counter, 1u) == (unsigned)nb - 1;
    __syncthreads();
    if (!s_last || warp != 0) return;
    __threadfence();
    double t = 0.0;
    for (int b = lane; b < nb; b += 32) t += __ldcg(a.blk + b);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    if (lane == 0) {
        *a.gn2_out = t;
        a.st->counter = 0u;
    }
}

__global__ void __launch_bounds__(AD_ITEMS* AD_WARPS) p2_adam_kernel(const P2AdamArgs a) {
    adam_body(a, blockIdx.x, gridDim.x);
}

// Batched markets: block j updates block bmap[j].y of market bmap[j].x (a.nblk blocks each).
__global__ void __launch_bounds__(AD_ITEMS* AD_WARPS)
    p2_adam_batch_kernel(const P2AdamArgs* __restrict__ aa, const int2* __restrict__ bmap) {
    const int2 mb = bmap[blockIdx.x];
    const P2AdamArgs a = aa[mb.x];
    adam_body(a, mb.y, a.nblk);
}

// Policy of consumers u0.. (one CTA each): x_ik = softmax_k(g^(L-1)'_k + s_i (e_k - e_max)),
// s_i = r(u,i) w_i / (eps ln 2), the policy of the last row update; public [u][i][k] layout.
__global__ void p2_policy_kernel(const P2Args a, int u0, float* __restrict__ x) {
    const int u = u0 + blockIdx.x;
    const int nc = a.nc;
    const float* gp = a.gP + (size_t)u * nc;
    for (int i = threadIdx.x; i < a.I; i += blockDim.x) {
        const size_t o = (size_t)u * a.ld + i;
        const float r = a.r_bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(a.r)[o])
                                 : static_cast<const float*>(a.r)[o];
        const float si = r * a.w[i] * a.inv_eps_ln2;
        float M = -INFINITY;
        for (int k = 0; k < nc; ++k) M = fmaxf(M, fmaf(si, a.e[k] - a.emax, gp[k]));
        float S = 0.f;
        for (int k = 0; k < nc; ++k) S += ex2(fmaf(si, a.e[k] - a.emax, gp[k]) - M);
        const float inv = 1.f / S;
        float* xo = x + ((size_t)blockIdx.x * a.I + i) * nc;
        for (int k = 0; k < nc; ++k) xo[k] = ex2(fmaf(si, a.e[k] - a.emax, gp[k]) - M) * inv;
    }
}

__global__ void exp_theta_kernel(const float* __restrict__ theta, float* __restrict__ w, int I,
                                 int ld) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ld; i += gridDim.x * blockDim.x)
        w[i] = i < I ? expf(theta[i]) : 0.f;
}

}  // namespace

int p2_adam_blocks(int I) { return (I + AD_ITEMS - 1) / AD_ITEMS; }

// Rows per thread: 8 for up to 1024 items, 16 up to 8192, 24 up to 12288 (CTA <= 512 threads);
// 21 columns take 20 up to 10240 items. Above 8192 items one CTA fills an SM (its per-item arrays),
// so the CTA's own warps are all the latency hiding there is: at 10^4 items 20 rows give 512
// threads (16 warps, 115 registers) against 448 for 24, and the Sinkhorn kernel ran 73.0 instead
// of 85.9 ms (the gradient kernel 19.9 instead of 22.0 ms) for 40000 consumers, L = 50.
bool p2_select(int nc, int I, P2Variant* out) {
    auto threads_for = [&](int R) {
        const int t = (I + R - 1) / R;
        return (t + 31) / 32 * 32;
    };
    int R = I <= 1024 ? 8 : (threads_for(16) <= 512 ? 16 : 24);
    if (R == 24 && nc == 21 && threads_for(20) <= 512) R = 20;
    if (threads_for(R) > 512) return false;
    const int T = threads_for(R);
    if (nc == 21) return p2_variant_k21(R, T, out);
    if (nc == 11) return p2_variant_k11(R, T, out);
    if (nc == 6) return p2_variant_k6(R, T, out);
    if (threads_for(8) > 512) return false;
    const int ncb = nc <= 8 ? 8 : (nc <= 16 ? 16 : (nc <= 32 ? 32 : 0));
    if (!ncb) return false;
    return p2_variant_generic(ncb, threads_for(8), out);
}

size_t p2_sweep_smem(const P2Variant& v, int nc, int ld, int esz) {
    return p2::sweep_layout(v.ncb, nc, ld, v.threads / 32, esz, nullptr, nullptr);
}

size_t p2_grad_smem(const P2Variant& v, int nc, int ld, int esz) {
    return p2::grad_layout(v.ncb, nc, ld, v.threads / 32, esz, nullptr, nullptr);
}

cudaError_t p2_launch_sweep(const P2Variant& v, const P2Args& a, cudaStream_t s) {
    void* args[] = {const_cast<P2Args*>(&a)};
    return cudaLaunchKernel(v.sweep, dim3(a.G), dim3(v.threads), args,
                            p2_sweep_smem(v, a.nc, a.ld, a.r_bf16 ? 2 : 4), s);
}

cudaError_t p2_launch_grad(const P2Variant& v, const P2Args& a, cudaStream_t s) {
    void* args[] = {const_cast<P2Args*>(&a)};
    return cudaLaunchKernel(v.grad, dim3(a.G), dim3(v.threads), args,
                            p2_grad_smem(v, a.nc, a.ld, a.r_bf16 ? 2 : 4), s);
}

size_t p2_sweep_smem_batch(const P2Variant& v, int ld_max, int esz) {
    return p2::sweep_layout(v.ncb, v.ncb, ld_max, v.threads / 32, esz, nullptr, nullptr);
}

size_t p2_grad_smem_batch(const P2Variant& v, int ld_max, int esz) {
    return p2::grad_layout(v.ncb, v.ncb, ld_max, v.threads / 32, esz, nullptr, nullptr);
}

cudaError_t p2_launch_sweep_batch(const P2Variant& v, const P2Batch& bt, int G, cudaStream_t s) {
    void* args[] = {const_cast<P2Batch*>(&bt)};
    return cudaLaunchKernel(v.sweep_b, dim3(G), dim3(v.threads), args,
                            p2_sweep_smem_batch(v, bt.ld_max, bt.esz), s);
}

cudaError_t p2_launch_grad_batch(const P2Variant& v, const P2Batch& bt, int G, cudaStream_t s) {
    void* args[] = {const_cast<P2Batch*>(&bt)};
    return cudaLaunchKernel(v.grad_b, dim3(G), dim3(v.threads), args,
                            p2_grad_smem_batch(v, bt.ld_max, bt.esz), s);
}

cudaError_t p2_launch_adam(const P2AdamArgs& a, cudaStream_t s) {
    p2_adam_kernel<<<p2_adam_blocks(a.I), AD_ITEMS * AD_WARPS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t p2_launch_adam_batch(const P2AdamArgs* aa, const int2* bmap, int nblocks, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    p2_adam_batch_kernel<<<nblocks, AD_ITEMS * AD_WARPS, 0, s>>>(aa, bmap);
    return cudaGetLastError();
}

cudaError_t launch_p2_policy(const P2Args& a, int u0, int n_u, float* x, cudaStream_t s) {
    if (n_u <= 0) return cudaSuccess;
    p2_policy_kernel<<<n_u, 256, 0, s>>>(a, u0, x);
    return cudaGetLastError();
}

cudaError_t launch_exp_theta(const float* theta, float* w, int I, int ld, cudaStream_t s) {
    exp_theta_kernel<<<(ld + 255) / 256, 256, 0, s>>>(theta, w, I, ld);
    return cudaGetLastError();
}

}  // namespace fr
