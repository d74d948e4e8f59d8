// fr_common.cu -- the cross-consumer impact reduction and the support kernels of libfairrank.
#include <cuda_bf16.h>

#include <cstring>

#include <mutex>

#include "fr_device.cuh"
#include "fr_internal.h"

namespace fr {

namespace {

constexpr int RED_ITEMS = 32;  // items per CTA (one per lane)
constexpr int RED_WARPS = 32;  // warps splitting the per-CTA partials
constexpr int RED_BATCH = 20;  // partial-row loads in flight per lane

// Eq. (4) across consumers and Eq. (5): Imp_i = sum over the sweep CTAs' partials (fixed order,
// compensated FP32 arithmetic carrying FP64-level precision, delivered as a double),
// omega_i = 1/Imp_i for the next gradient, F = sum_i log Imp_i in FP64. The last CTA to
// finish (atomic ticket) combines the per-CTA partial sums of log Imp_i, of Imp_i (utility,
// Sec. 4.1) and of the squared gradient norm in a fixed order, updates the step state and, for
// fr_solve, raises the stop flag once the step's gradient norm is <= the threshold.
// bid / nb: this CTA's index among the nb CTAs that reduce one problem.
__device__ __forceinline__ void reduce_body(const ReduceArgs& a, int bid, int nb) {
    __shared__ float2 s_sum[RED_WARPS][RED_ITEMS];  // per warp and item: compensated sum (s, c)
    __shared__ int s_last;
    if (a.st->stop) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int item = bid * RED_ITEMS + lane;
    // Knuth's TwoSum: t = s + x and the rounding error of that addition, carried exactly in c
    auto two_sum = [](float& s, float& c, float x) {
        const float t = __fadd_rn(s, x);
        const float bp = __fsub_rn(t, s);
        c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
        s = t;
    };
    // partials g = warp, warp + RED_WARPS, ... in two interleaved compensated FP32 sums, so each
    // warp's total s + c is accurate to double-level precision without FP64 arithmetic per partial
    // (the FP64 pipe is a small fraction of the FP32 one on this part); the fixed order keeps it
    // deterministic
    float sa[2] = {0.f, 0.f}, ca[2] = {0.f, 0.f};
    if (item < a.I) {
        const float* p = a.part + item;
        const size_t step = (size_t)RED_WARPS * a.ld;
        int g = warp;
        // RED_BATCH loads in flight per lane: up to 640 partial rows (a grid of 4 CTAs per SM) take
        // one round trip to L2; RED_BATCH is even, so every row keeps its accumulator (j & 1)
        for (; g + (RED_BATCH - 1) * RED_WARPS < a.G; g += RED_BATCH * RED_WARPS) {
            const float* q = p + (size_t)g * a.ld;
            float x[RED_BATCH];
#pragma unroll
            for (int j = 0; j < RED_BATCH; ++j) x[j] = __ldcg(q + j * step);
#pragma unroll
            for (int j = 0; j < RED_BATCH; ++j) two_sum(sa[j & 1], ca[j & 1], x[j]);
        }
        {  // the remaining fewer than RED_BATCH, all loads first (zeros add exactly)
            float x[RED_BATCH];
#pragma unroll
            for (int j = 0; j < RED_BATCH; ++j)
                x[j] = g + j * RED_WARPS < a.G ? __ldcg(p + (size_t)(g + j * RED_WARPS) * a.ld) : 0.f;
#pragma unroll
            for (int j = 0; j < RED_BATCH; ++j) two_sum(sa[j & 1], ca[j & 1], x[j]);
        }
    }
    // the two accumulators and then the warps combined as double-float pairs (s, c): s absorbs the
    // other's s by TwoSum, the rounding error and both c's go to c; warps pairwise in a fixed tree
    two_sum(sa[0], ca[0], sa[1]);
    ca[0] = __fadd_rn(ca[0], ca[1]);
    s_sum[warp][lane] = make_float2(sa[0], ca[0]);
#pragma unroll
    for (int h = RED_WARPS / 2; h > 0; h >>= 1) {
        __syncthreads();
        if (warp < h) {
            const float2 o = s_sum[warp + h][lane];
            float ss = s_sum[warp][lane].x, cc = s_sum[warp][lane].y;
            two_sum(ss, cc, o.x);
            cc = __fadd_rn(cc, o.y);
            s_sum[warp][lane] = make_float2(ss, cc);
        }
    }
    if (warp == 0) {
        const float2 t2 = s_sum[0][lane];
        const double tot = (double)t2.x + (double)t2.y;
        double lg = 0.0, im = 0.0;
        if (item < a.I) {
            a.imp[item] = tot;
            a.omega[item] = (float)(1.0 / tot);
            if (!(tot > 0.0) || !isfinite(tot)) atomicOr(&a.st->err, 1);
            lg = log(tot);
            im = tot;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lg += __shfl_xor_sync(FULL, lg, o);
            im += __shfl_xor_sync(FULL, im, o);
        }
        if (lane == 0) {
            a.blk[2 * bid] = lg;
            a.blk[2 * bid + 1] = im;
        }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(&a.st->counter, 1u) == (unsigned)nb - 1;
    __syncthreads();
    if (!s_last || warp != 0) return;
    __threadfence();
    double F = 0.0, S = 0.0, g2 = 0.0;
    for (int b = lane; b < nb; b += 32) {
        F += __ldcg(a.blk + 2 * b);
        S += __ldcg(a.blk + 2 * b + 1);
    }
    if (a.after_update) {  // partials lane, lane + 32, ... in that order, RED_BATCH loads in flight
        for (int g0 = 0; g0 < a.Ggn; g0 += 32 * RED_BATCH) {
            double y[RED_BATCH];
#pragma unroll
            for (int j = 0; j < RED_BATCH; ++j) {
                const int g = g0 + lane + 32 * j;
                y[j] = g < a.Ggn ? __ldcg(a.gn2_part + g) : 0.0;
            }
#pragma unroll
            for (int j = 0; j < RED_BATCH; ++j)
                if (g0 + lane + 32 * j < a.Ggn) g2 += y[j];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        F += __shfl_xor_sync(FULL, F, o);
        S += __shfl_xor_sync(FULL, S, o);
        g2 += __shfl_xor_sync(FULL, g2, o);
    }
    if (lane == 0) {
        DevState* st = a.st;
        st->F = F;
        st->utility = S / a.U;
        if (!isfinite(F)) st->err |= 1;
        if (a.after_update) {
            const double gn = sqrt(g2);
            if (!isfinite(gn)) st->err |= 2;
            st->gnorm = gn;
            st->t += 1;
            st->steps_done += 1;
            const int h = st->hist_idx;
            if (h < a.hist_cap) {
                a.F_hist[h] = F;
                a.gn_hist[h] = gn;
            }
            st->hist_idx = h + 1;
            if (st->thresh >= 0.0 && gn <= st->thresh) st->stop = 1;
            if (st->max_steps > 0 && st->steps_done >= st->max_steps) st->stop = 1;
        }
        st->counter = 0u;
    }
}

__global__ void __launch_bounds__(RED_ITEMS* RED_WARPS) reduce_kernel(const ReduceArgs a) {
    reduce_body(a, blockIdx.x, gridDim.x);
}

// Batched markets: block j reduces block bmap[j].y of market bmap[j].x (a.nblk blocks each).
__global__ void __launch_bounds__(RED_ITEMS* RED_WARPS)
    reduce_batch_kernel(const ReduceArgs* __restrict__ ra, const int2* __restrict__ bmap) {
    const int2 mb = bmap[blockIdx.x];
    const ReduceArgs a = ra[mb.x];
    reduce_body(a, mb.y, a.nblk);
}

// [U][I][nc] -> [U][nc][ld] (padding rows zero), times scale
__global__ void pack_kernel(const float* __restrict__ src, float* __restrict__ dst, int U, int I,
                            int nc, int ld, float scale) {
    const long long n = (long long)U * nc * ld;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(j % ld);
        const long long uk = j / ld;
        const int k = (int)(uk % nc);
        const long long u = uk / nc;
        dst[j] = i < I ? src[(u * I + i) * nc + k] * scale : 0.f;
    }
}

__global__ void unpack_kernel(const float* __restrict__ src, float* __restrict__ dst, int U, int I,
                              int nc, int ld, float scale) {
    const long long n = (long long)U * I * nc;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(j % nc);
        const long long ui = j / nc;
        const int i = (int)(ui % I);
        const long long u = ui / I;
        dst[j] = src[(u * nc + k) * ld + i] * scale;
    }
}

__global__ void scale_kernel(const float* __restrict__ src, float* __restrict__ dst, long long n,
                             float scale) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x)
        dst[j] = src[j] * scale;
}

__global__ void relevance_import_kernel(const void* __restrict__ src, int dtype, long long ld_src,
                                        void* __restrict__ dst, int dst_bf16, int U, int I, int ld) {
    const long long n = (long long)U * ld;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(j % ld);
        const long long u = j / ld;
        float v = 0.f;
        if (i < I) {
            const long long o = u * ld_src + i;
            if (dtype == FR_F32) v = static_cast<const float*>(src)[o];
            else if (dtype == FR_F64) v = (float)static_cast<const double*>(src)[o];
            else v = __bfloat162float(static_cast<const __nv_bfloat16*>(src)[o]);
        }
        if (dst_bf16)
            static_cast<__nv_bfloat16*>(dst)[j] = __float2bfloat16_rn(v);
        else
            static_cast<float*>(dst)[j] = v;
    }
}

// flags[0] |= 1 for a negative or non-finite value; flags[1] counts items without positive r.
// Block b checks items 32 b .. 32 b + 31 (one per lane, 128-byte row segments); its warps split the
// consumers, and a shared flag per item collects whether any consumer's relevance is positive.
__global__ void __launch_bounds__(1024) relevance_check_kernel(const void* __restrict__ r, int r_bf16,
                                                               int U, int I, int ld, int* flags) {
    __shared__ int s_pos[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    if (threadIdx.x < 32) s_pos[threadIdx.x] = 0;
    __syncthreads();
    bool bad = false, pos = false;
    if (i < I) {
        for (int u = warp; u < U; u += W) {
            const size_t o = (size_t)u * ld + i;
            const float v = r_bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(r)[o])
                                   : static_cast<const float*>(r)[o];
            bad |= !(v >= 0.f) || !isfinite(v);
            pos |= v > 0.f;
        }
    }
    if (pos) atomicOr(&s_pos[lane], 1);
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(flags, 1);
    __syncthreads();
    if (warp == 0 && i < I && !s_pos[lane]) atomicAdd(flags + 1, 1);
}

// Policy of consumers u0.. (one CTA each): x_ik = softmax_k(g^(L-1)'_k - c'_ik) in base 2, the
// policy emitted by the last Sinkhorn row update; written in the public [u][i][k] layout.
__global__ void policy_kernel(const P1Args a, int u0, float* __restrict__ x) {
    const int u = u0 + blockIdx.x;
    const int nc = a.nc;
    const float* C = a.C + (size_t)u * nc * a.ld;
    const float* gp = a.gP + (size_t)u * nc;
    for (int i = threadIdx.x; i < a.I; i += blockDim.x) {
        float M = -INFINITY;
        for (int k = 0; k < nc; ++k) M = fmaxf(M, gp[k] - C[(size_t)k * a.ld + i] * a.inv_eps_ln2);
        float S = 0.f;
        for (int k = 0; k < nc; ++k) S += ex2(gp[k] - C[(size_t)k * a.ld + i] * a.inv_eps_ln2 - M);
        const float inv = 1.f / S;
        float* xo = x + ((size_t)blockIdx.x * a.I + i) * nc;
        for (int k = 0; k < nc; ++k)
            xo[k] = ex2(gp[k] - C[(size_t)k * a.ld + i] * a.inv_eps_ln2 - M) * inv;
    }
}

// 8 independent chains x <- 2^(-x) per thread: MUFU-bound throughput probe
__global__ void ex2_bench_kernel(float* sink, int iters) {
    float x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = 0.1f * j + 1e-3f * (threadIdx.x & 31);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = ex2(-x[j]);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += x[j];
    if (s == 12345.f) sink[blockIdx.x] = s;
}

// ---- on-chip peak probes (fr_measure_peaks) ------------------------------------------------------
// Block 0's thread 0 records the SM clock and the global timer around its loop (clk[0..1]: cycles,
// nanoseconds), which gives the clock the SMs ran at during the probe.

// Shared-memory load bandwidth: every thread loads VB-byte vectors (8 or 16) from consecutive
// addresses (conflict-free, the sweeps' access pattern), eight independent loads per iteration,
// with the offset advanced each iteration so that no load can be hoisted; the loaded values are
// summed with packed adds so that they are used.
template <int VB>
__global__ void smem_bench_kernel(float* sink, int iters, unsigned long long* clk) {
    extern __shared__ __align__(16) float sbuf[];  // 16 KB
    constexpr int NF = 16384 / 4;
    for (int i = threadIdx.x; i < NF; i += blockDim.x) sbuf[i] = 1e-3f * (i & 63);
    __syncthreads();
    const unsigned base = (unsigned)__cvta_generic_to_shared(sbuf);
    constexpr unsigned span = 16384u;
    unsigned off = (unsigned)(threadIdx.x * VB) % span;
    f2 acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0ull;
    unsigned long long c0 = 0, t0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c0 = clock64();
        t0 = global_ns();
    }
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const unsigned a = base + ((off + (unsigned)j * 1024u * VB / 8u) & (span - 1u));
            if constexpr (VB == 8) {
                f2 v;
                asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(a));
                acc[j] = add2(acc[j], v);
            } else {
                f2 v0, v1;
                asm volatile("ld.shared.v2.b64 {%0, %1}, [%2];" : "=l"(v0), "=l"(v1) : "r"(a));
                acc[j] = add2(acc[j], add2(v0, v1));
            }
        }
        off = (off + 32u * VB) & (span - 1u);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        clk[0] = clock64() - c0;
        clk[1] = global_ns() - t0;
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float a, b;
        upk(acc[j], a, b);
        s += a + b;
    }
    if (s == 12345.f) sink[blockIdx.x] = s;
}

// FP32 fused multiply-add rate: eight independent chains per thread, scalar (PACKED = false) or
// packed f32x2 (each instruction two multiply-adds).
template <bool PACKED>
__global__ void fma_bench_kernel(float* sink, int iters, unsigned long long* clk) {
    unsigned long long c0 = 0, t0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c0 = clock64();
        t0 = global_ns();
    }
    float s = 0.f;
    if constexpr (PACKED) {
        f2 x[8];
        const f2 m = pk(0.999f, 0.998f), c = pk(1e-3f, 2e-3f);
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = pk(0.1f * j, 1e-3f * (threadIdx.x & 31));
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < 8; ++j) x[j] = fma2(x[j], m, c);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float a, b;
            upk(x[j], a, b);
            s += a + b;
        }
    } else {
        float x[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] = 0.1f * j + 1e-3f * (threadIdx.x & 31);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int j = 0; j < 8; ++j) x[j] = fmaf(x[j], 0.999f, 1e-3f);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) s += x[j];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        clk[0] = clock64() - c0;
        clk[1] = global_ns() - t0;
    }
    if (s == 12345.f) sink[blockIdx.x] = s;
}

__global__ void solve_cond_kernel(const DevState* st, int* ctl, cudaGraphConditionalHandle h) {
    const int it = ctl[0] + 1;
    ctl[0] = it;
    const bool more = st->stop == 0 && st->err == 0 && it < ctl[1];
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

}  // namespace

int reduce_blocks(int I) { return (I + RED_ITEMS - 1) / RED_ITEMS; }

cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    if ((size_t)fa.maxDynamicSharedSizeBytes >= bytes) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t reduce_launch(const ReduceArgs& a, cudaStream_t s) {
    reduce_kernel<<<reduce_blocks(a.I), RED_ITEMS * RED_WARPS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t reduce_launch_batch(const ReduceArgs* ra, const int2* bmap, int nblocks, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    reduce_batch_kernel<<<nblocks, RED_ITEMS * RED_WARPS, 0, s>>>(ra, bmap);
    return cudaGetLastError();
}

cudaError_t launch_pack_ikn_to_kni(const float* src, float* dst, int U, int I, int nc, int ld,
                                   float scale, cudaStream_t s) {
    pack_kernel<<<grid_for((long long)U * nc * ld), 256, 0, s>>>(src, dst, U, I, nc, ld, scale);
    return cudaGetLastError();
}

cudaError_t launch_unpack_kni_to_ikn(const float* src, float* dst, int U, int I, int nc, int ld,
                                     float scale, cudaStream_t s) {
    unpack_kernel<<<grid_for((long long)U * I * nc), 256, 0, s>>>(src, dst, U, I, nc, ld, scale);
    return cudaGetLastError();
}

cudaError_t launch_scale(const float* src, float* dst, long long n, float scale, cudaStream_t s) {
    scale_kernel<<<grid_for(n), 256, 0, s>>>(src, dst, n, scale);
    return cudaGetLastError();
}

cudaError_t launch_relevance_import(const void* src, int dtype, long long ld_src, void* dst,
                                    int dst_bf16, int U, int I, int ld, cudaStream_t s) {
    relevance_import_kernel<<<grid_for((long long)U * ld), 256, 0, s>>>(src, dtype, ld_src, dst,
                                                                         dst_bf16, U, I, ld);
    return cudaGetLastError();
}

cudaError_t launch_relevance_check(const void* r, int r_bf16, int U, int I, int ld, int* flags,
                                   cudaStream_t s) {
    relevance_check_kernel<<<(I + 31) / 32, 1024, 0, s>>>(r, r_bf16, U, I, ld, flags);
    return cudaGetLastError();
}

cudaError_t launch_policy(const P1Args& a, int u0, int n_u, float* x_out, cudaStream_t s) {
    if (n_u <= 0) return cudaSuccess;
    policy_kernel<<<n_u, 256, 0, s>>>(a, u0, x_out);
    return cudaGetLastError();
}

cudaError_t launch_solve_cond(const DevState* st, int* ctl, cudaGraphConditionalHandle h,
                              cudaStream_t s) {
    solve_cond_kernel<<<1, 1, 0, s>>>(st, ctl, h);
    return cudaGetLastError();
}

cudaError_t launch_ex2_bench(float* sink, int blocks, int threads, int iters, cudaStream_t s) {
    ex2_bench_kernel<<<blocks, threads, 0, s>>>(sink, iters);
    return cudaGetLastError();
}

// ---- self-check of the column update's log2 (fr_check_log2_near1) -------------------------------
// Every float y with |y - 1| < 2^-5 (the range of the short path), as consecutive bit patterns from
// start: the relative error of log2_near1(y) and of log2f(y) against log2 in double precision,
// maxima kept as the bit patterns of non-negative floats (which order like the floats); y = 1 must
// give exactly 0 (counted in bad).
__global__ void log2_check_kernel(unsigned start, unsigned count, unsigned* out) {
    unsigned m_near = 0u, m_lib = 0u, bad = 0u;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < count; k += gridDim.x * blockDim.x) {
        const float y = __uint_as_float(start + k);
        const float a = log2_near1(y), b = log2f(y);
        const double ex = log2((double)y);
        if (ex == 0.0) {
            bad += a != 0.f;
            continue;
        }
        m_near = max(m_near, __float_as_uint((float)fabs(((double)a - ex) / ex)));
        m_lib = max(m_lib, __float_as_uint((float)fabs(((double)b - ex) / ex)));
    }
    atomicMax(out, m_near);
    atomicMax(out + 1, m_lib);
    if (bad) atomicAdd(out + 2, bad);
}

static unsigned host_bits(float x) {
    unsigned u;
    std::memcpy(&u, &x, sizeof u);
    return u;
}

cudaError_t launch_log2_check(unsigned* out, int blocks, cudaStream_t s) {
    const unsigned lo = host_bits(1.f - 0x1p-5f) + 1u;  // first float above 1 - 2^-5
    const unsigned hi = host_bits(1.f + 0x1p-5f) - 1u;  // last float below 1 + 2^-5
    log2_check_kernel<<<blocks, 256, 0, s>>>(lo, hi - lo + 1u, out);
    return cudaGetLastError();
}

cudaError_t launch_peak_bench(int kind, float* sink, int blocks, int threads, int iters,
                              unsigned long long* clk, cudaStream_t s) {
    switch (kind) {
        case 0: smem_bench_kernel<8><<<blocks, threads, 16384, s>>>(sink, iters, clk); break;
        case 1: smem_bench_kernel<16><<<blocks, threads, 16384, s>>>(sink, iters, clk); break;
        case 2: fma_bench_kernel<false><<<blocks, threads, 0, s>>>(sink, iters, clk); break;
        default: fma_bench_kernel<true><<<blocks, threads, 0, s>>>(sink, iters, clk); break;
    }
    return cudaGetLastError();
}

}  // namespace fr
