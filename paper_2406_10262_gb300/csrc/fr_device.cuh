// fr_device.cuh -- small device helpers shared by the libfairrank kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fr {

constexpr unsigned FULL = 0xffffffffu;

// 2^x on the multi-function unit (one MUFU.EX2); flushes subnormal results to zero.
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/x on the multi-function unit (relative error below 2^-22 over the normal range).
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// log2(x) on the multi-function unit (absolute error ~2^-22 near 1).
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Smallest power of two >= n (1 for n <= 1). A loop, not a recursion: called with a run-time
// argument (the shared-memory layouts), a recursive device function stays an out-of-line call
// whose frames the compiler's per-thread stack size does not include, so a kernel whose own frame
// is close to the stack limit would overrun it.
__host__ __device__ __forceinline__ constexpr int pow2ceil(int n) {
    int p = 1;
    while (p < n) p *= 2;
    return p;
}

// Adam's bias correction 1 - beta^t (beta in [0.5, 1), t >= 1) in FP32 without cancellation, as
// -expm1(t log1p(beta - 1)): beta - 1 is exact, and the result keeps a few-ulp relative accuracy
// where 1 - powf(beta, t) would lose log2(1 / (1 - beta)) bits. (The double-precision pow it
// replaces is a long sequence on the FP64 pipe, and one thread's evaluation held its CTA.)
__device__ __forceinline__ float one_minus_pow(float beta, float t) {
    return -expm1f(t * log1pf(beta - 1.f));
}

// ---- bulk (TMA) copies and mbarriers --------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// Global -> shared bulk copy completing on `bar` (16-byte aligned addresses, size % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Bulk prefetch of [src, src + bytes) into L2 (16-byte aligned, size % 16 == 0).
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// Bounded wait for phase `parity` of `bar`: returns false if it did not complete within
// `max_polls` polls (the caller records an error instead of spinning forever).
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          unsigned max_polls) {
    for (unsigned it = 0; it < max_polls; ++it) {
        unsigned done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Nanoseconds of the global timer.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait of every thread of a CTA for phase `parity` of `bar` (a staged bulk copy), with one
// outcome for the whole CTA: true if every thread saw the phase complete within `max_polls` polls.
// Otherwise thread 0 sets `flag` in *err and every thread waits again, with `drain_polls`, for the
// copy to land, so that the caller can stop without a bulk copy still writing into this CTA's
// shared memory; the result is then false in every thread. Contains one __syncthreads_or (which
// also makes the caller's earlier shared-memory writes visible); every thread must call it.
__device__ __forceinline__ bool cta_wait_or_drain(unsigned long long* bar, unsigned parity,
                                                  unsigned max_polls, unsigned drain_polls,
                                                  int* err, int flag) {
    const bool ok = mbar_wait(bar, parity, max_polls);
    if (!__syncthreads_or(!ok)) return true;
    if (threadIdx.x == 0) atomicOr(err, flag);
    mbar_wait(bar, parity, drain_polls);
    return false;
}

// ---- packed pairs of FP32 values (sm_100+ f32x2 arithmetic: two lanes per instruction) ---------
typedef unsigned long long f2;

__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1,%2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float& a, float& b) {
    asm("mov.b64 {%0,%1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---- vector loads/stores of R consecutive floats (R in {1,2,4,8}; 4R-byte aligned) ------------
template <int R>
__device__ __forceinline__ void ldv(float (&d)[R], const float* p) {
    if constexpr (R == 1) {
        d[0] = *p;
    } else if constexpr (R == 2) {
        float2 v = *reinterpret_cast<const float2*>(p);
        d[0] = v.x; d[1] = v.y;
    } else if constexpr (R == 4) {
        float4 v = *reinterpret_cast<const float4*>(p);
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
    } else if constexpr (R == 6) {  // 24-byte stride: three 8-byte loads
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float2 v = reinterpret_cast<const float2*>(p)[j];
            d[2 * j] = v.x; d[2 * j + 1] = v.y;
        }
    } else {
        static_assert(R == 8, "R");
        float4 v = reinterpret_cast<const float4*>(p)[0];
        float4 w = reinterpret_cast<const float4*>(p)[1];
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
        d[4] = w.x; d[5] = w.y; d[6] = w.z; d[7] = w.w;
    }
}

template <int R>
__device__ __forceinline__ void stv(float* p, const float (&d)[R]) {
    if constexpr (R == 1) {
        *p = d[0];
    } else if constexpr (R == 2) {
        *reinterpret_cast<float2*>(p) = make_float2(d[0], d[1]);
    } else if constexpr (R == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(d[0], d[1], d[2], d[3]);
    } else if constexpr (R == 6) {
#pragma unroll
        for (int j = 0; j < 3; ++j) reinterpret_cast<float2*>(p)[j] = make_float2(d[2 * j], d[2 * j + 1]);
    } else {
        static_assert(R == 8, "R");
        reinterpret_cast<float4*>(p)[0] = make_float4(d[0], d[1], d[2], d[3]);
        reinterpret_cast<float4*>(p)[1] = make_float4(d[4], d[5], d[6], d[7]);
    }
}

// ---- warp reduce-scatter ------------------------------------------------------------------
// Each lane holds P values (P a power of two). After the call the lanes with owner == true hold,
// in v[0 .. max(P/32,1)), the warp-wide sums of columns base, base+1, ...; every column has
// exactly one owner. Costs P/2 + P/4 + ... shuffles instead of 5P for P separate butterflies.
template <int n, int o>
__device__ __forceinline__ void rs_level(float* v, int lane, int& base, bool& owner) {
    if constexpr (n == 1) {  // one value left: plain butterfly, the lower lane owns the sum
        v[0] += __shfl_xor_sync(FULL, v[0], o);
        if (lane & o) owner = false;
    } else {
        constexpr int h = n / 2;
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < h; ++j) {
            const float a = v[j], b = v[h + j];
            const float send = hi ? a : b;
            const float keep = hi ? b : a;
            v[j] = keep + __shfl_xor_sync(FULL, send, o);
        }
        if (hi) base += h;
    }
}

template <int P>
__device__ __forceinline__ int warp_reduce_scatter(float* v, int lane, bool& owner) {
    static_assert((P & (P - 1)) == 0, "power of two");
    int base = 0;
    owner = true;
    constexpr int n0 = P, n1 = n0 > 1 ? n0 / 2 : 1, n2 = n1 > 1 ? n1 / 2 : 1,
                  n3 = n2 > 1 ? n2 / 2 : 1, n4 = n3 > 1 ? n3 / 2 : 1;
    rs_level<n0, 16>(v, lane, base, owner);
    rs_level<n1, 8>(v, lane, base, owner);
    rs_level<n2, 4>(v, lane, base, owner);
    rs_level<n3, 2>(v, lane, base, owner);
    rs_level<n4, 1>(v, lane, base, owner);
    return base;
}

// Sum of NV per-thread vectors of length NCB over the whole CTA into out[j*ncp + k] (k < nc).
// s_red needs (blockDim/32) * NV * pow2ceil(NCB) floats. Deterministic (fixed order). Contains two
// __syncthreads; every thread of the CTA must call it.
template <int NCB, int NV>
__device__ __forceinline__ void cta_reduce(float (&v)[NV][NCB], int nc, float* s_red, float* out,
                                           int ncp) {
    constexpr int P = pow2ceil(NCB);
    constexpr int PER = P >= 32 ? P / 32 : 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        float w[P];
#pragma unroll
        for (int k = 0; k < P; ++k) w[k] = k < NCB ? v[j][k] : 0.f;
        bool owner;
        const int base = warp_reduce_scatter<P>(w, lane, owner);
        if (owner) {
#pragma unroll
            for (int q = 0; q < PER; ++q) {
                const int k = base + q;
                if (k < nc) s_red[(warp * NV + j) * P + k] = w[q];
            }
        }
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < NV * nc; idx += blockDim.x) {
        const int j = idx / nc, k = idx - j * nc;
        float s = 0.f;
        for (int ww = 0; ww < W; ++ww) s += s_red[(ww * NV + j) * P + k];
        out[j * ncp + k] = s;
    }
    __syncthreads();
}

// Sum of one per-thread vector of length N over the CTA into out[k] (k < n_valid). s_red needs
// (blockDim/32) * pow2ceil(N) floats. Deterministic; two __syncthreads.
template <int N>
__device__ __forceinline__ void cta_reduce_vec(float (&v)[N], int n_valid, float* s_red, float* out) {
    constexpr int P = pow2ceil(N);
    constexpr int PER = P >= 32 ? P / 32 : 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    float w[P];
#pragma unroll
    for (int k = 0; k < P; ++k) w[k] = k < N ? v[k] : 0.f;
    bool owner;
    const int base = warp_reduce_scatter<P>(w, lane, owner);
    if (owner) {
#pragma unroll
        for (int q = 0; q < PER; ++q)
            if (base + q < n_valid) s_red[warp * P + base + q] = w[q];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n_valid; k += blockDim.x) {
        float s = 0.f;
        for (int ww = 0; ww < W; ++ww) s += s_red[ww * P + k];
        out[k] = s;
    }
    __syncthreads();
}

// ---- pieces shared by the Sinkhorn kernels --------------------------------------------------

// Cholesky solve of the n x n SPD system A (row-major) with right-hand side rhs, by one warp, in
// double precision (wide tiles). Pivots below `floor` are raised to it (a column with no mass
// leaves the Laplacian-like Gram matrix singular; its beta is then ~0).
__device__ inline void warp_cholesky_solve(double* A, double* rhs, int n, int lane) {
    double dmax = 0.0;
    for (int j = 0; j < n; ++j) dmax = fmax(dmax, A[j * n + j]);
    const double floor_ = 1e-13 * fmax(dmax, 1e-300);
    for (int j = 0; j < n; ++j) {
        __syncwarp();
        const double ljj = sqrt(fmax(A[j * n + j], floor_));
        for (int i = j + 1 + lane; i < n; i += 32) A[i * n + j] /= ljj;
        __syncwarp();
        if (lane == 0) A[j * n + j] = ljj;
        const int m = n - j - 1;
        for (int idx = lane; idx < m * m; idx += 32) {
            const int i = j + 1 + idx / m, k = j + 1 + idx % m;
            if (k <= i) A[i * n + k] -= A[i * n + j] * A[k * n + j];
        }
    }
    __syncwarp();
    for (int j = 0; j < n; ++j) {  // L y = rhs
        const double yj = rhs[j] / A[j * n + j];
        __syncwarp();
        for (int i = j + 1 + lane; i < n; i += 32) rhs[i] -= A[i * n + j] * yj;
        if (lane == 0) rhs[j] = yj;
        __syncwarp();
    }
    for (int j = n - 1; j >= 0; --j) {  // L^T z = y
        const double zj = rhs[j] / A[j * n + j];
        __syncwarp();
        for (int i = lane; i < j; i += 32) rhs[i] -= A[j * n + i] * zj;
        if (lane == 0) rhs[j] = zj;
        __syncwarp();
    }
}

// Solve of the n x n SPD system (n <= NM <= 31) held in shared memory (A row-major, rhs), by one
// warp in single precision: lane i keeps row i of A in registers; right-looking Cholesky with the
// pivot column broadcast by shuffles, forward substitution in registers, back substitution from a
// transposed copy of L in shared memory (Lt, n*n floats). Pivots below `floor` are raised to it.
// Each pivot costs one reciprocal square root (rsqrt.approx) and the divisions by L_jj become
// multiplications by it: the n pivots form a sequential chain, and IEEE square root and division
// are long software sequences. Two forms with the same arithmetic (bit-identical results): up to 12
// unknowns the pivot and substitution loops stay rolled (the pivot's row entry picked from the
// registers by a select chain) -- the solve runs once per consumer between long sweeps, and the
// fully unrolled straight-line form cost 2 % more of the fused 11-column step; for wider systems
// the select chains and full-width shuffles of the rolled form grow with n, and the unrolled form
// (shuffles only for the trailing columns) is 3 % faster in the 21-column per-item gradient.
// Writes beta[0..n).
template <int NM>
__device__ inline void warp_cholesky_solve_f32_rolled(const float* A, const float* rhs, int n,
                                                      float* Lt, float* beta, int lane) {
    float row[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) row[k] = (lane < n && k < n) ? A[lane * n + k] : 0.f;
    float dmax = 0.f;
#pragma unroll 1
    for (int j = 0; j < n; ++j) dmax = fmaxf(dmax, A[j * n + j]);
    const float floor_ = 1e-12f * fmaxf(dmax, 1e-30f);
    float rinv = 0.f;  // lane j: 1 / L_jj
#pragma unroll 1
    for (int j = 0; j < n; ++j) {
        float rj = row[0];  // row[j]
#pragma unroll
        for (int k = 1; k < NM; ++k) rj = k == j ? row[k] : rj;
        const float d = fmaxf(__shfl_sync(FULL, rj, j), floor_);
        const float ri = rsqrtf(d);
        const float lij = lane > j ? rj * ri : (lane == j ? d * ri : 0.f);
        if (lane == j) rinv = ri;
#pragma unroll
        for (int k = 0; k < NM; ++k) {
            if (k == j) row[k] = lij;
            const float lkj = __shfl_sync(FULL, lij, k);
            if (k > j && lane > j) row[k] = fmaf(-lij, lkj, row[k]);
        }
    }
    float y = lane < n ? rhs[lane] : 0.f;  // L y = rhs: lane i holds y_i
#pragma unroll 1
    for (int j = 0; j < n; ++j) {
        float lj = row[0];  // L[lane][j]
#pragma unroll
        for (int k = 1; k < NM; ++k) lj = k == j ? row[k] : lj;
        const float yj = __shfl_sync(FULL, y * rinv, j);
        if (lane == j) y = yj;
        if (lane > j) y = fmaf(-lj, yj, y);
    }
    if (lane < n) {  // Lt[k][i] = L[i][k]
#pragma unroll
        for (int k = 0; k < NM; ++k)
            if (k < n) Lt[k * n + lane] = row[k];
    }
    __syncwarp();
    float z = y;  // L^T z = y
    for (int j = n - 1; j >= 0; --j) {
        const float zj = __shfl_sync(FULL, z * rinv, j);
        if (lane == j) z = zj;
        if (lane < j) z = fmaf(-Lt[lane * n + j], zj, z);  // (L^T)[i][j] = L[j][i]
    }
    if (lane < n) beta[lane] = z;
}

template <int NM>
__device__ inline void warp_cholesky_solve_f32_unrolled(const float* A, const float* rhs, int n,
                                                        float* Lt, float* beta, int lane) {
    float row[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) row[k] = (lane < n && k < n) ? A[lane * n + k] : 0.f;
    float dmax = 0.f;
#pragma unroll
    for (int j = 0; j < NM; ++j)
        if (j < n) dmax = fmaxf(dmax, __shfl_sync(FULL, row[j], j));
    const float floor_ = 1e-12f * fmaxf(dmax, 1e-30f);
    float rinv = 0.f;  // lane j: 1 / L_jj
#pragma unroll
    for (int j = 0; j < NM; ++j) {
        if (j >= n) break;
        const float d = fmaxf(__shfl_sync(FULL, row[j], j), floor_);
        const float ri = rsqrtf(d);
        const float lij = lane > j ? row[j] * ri : (lane == j ? d * ri : 0.f);
        if (lane == j) rinv = ri;
        row[j] = lij;
#pragma unroll
        for (int k = j + 1; k < NM; ++k) {
            const float lkj = __shfl_sync(FULL, lij, k);
            if (lane > j) row[k] = fmaf(-lij, lkj, row[k]);
        }
    }
    float y = lane < n ? rhs[lane] : 0.f;  // L y = rhs: lane i holds y_i
#pragma unroll
    for (int j = 0; j < NM; ++j) {
        if (j >= n) break;
        const float yj = __shfl_sync(FULL, y * rinv, j);
        if (lane == j) y = yj;
        if (lane > j) y = fmaf(-row[j], yj, y);
    }
    if (lane < n) {  // Lt[k][i] = L[i][k]
#pragma unroll
        for (int k = 0; k < NM; ++k)
            if (k < n) Lt[k * n + lane] = row[k];
    }
    __syncwarp();
    float z = y;  // L^T z = y
    for (int j = n - 1; j >= 0; --j) {
        const float zj = __shfl_sync(FULL, z * rinv, j);
        if (lane == j) z = zj;
        if (lane < j) z = fmaf(-Lt[lane * n + j], zj, z);  // (L^T)[i][j] = L[j][i]
    }
    if (lane < n) beta[lane] = z;
}

template <int NM>
__device__ inline void warp_cholesky_solve_f32(const float* A, const float* rhs, int n, float* Lt,
                                               float* beta, int lane) {
    if constexpr (NM <= 12)
        warp_cholesky_solve_f32_rolled<NM>(A, rhs, n, Lt, beta, lane);
    else
        warp_cholesky_solve_f32_unrolled<NM>(A, rhs, n, Lt, beta, lane);
}

// Broadcast of the column potentials held by lane k % 32 (slot k / 32) to every lane.
template <int NCB, int GPL>
__device__ __forceinline__ void bcast_g(const float (&gm)[GPL], float (&gk)[NCB]) {
#pragma unroll
    for (int k = 0; k < NCB; ++k) gk[k] = __shfl_sync(FULL, gm[k / 32], k % 32);
}

// log2(y) for y > 0, with a short path near 1, where the column updates of a converging Sinkhorn
// solve spend almost all their calls: for |y - 1| < 2^-5, t = y - 1 is exact and log2(1 + t) is
// the Taylor series of ln(1 + t) / ln 2 through t^6 in Horner form (truncation below 2^-30
// relative), a few dependent FMAs on the iteration's critical path; elsewhere log2f.
__device__ __forceinline__ float log2_near1(float y) {
    const float t = y - 1.f;
    if (fabsf(t) < 0x1p-5f) {
        constexpr float c1 = 1.4426950408889634f;    //  1 / ln 2
        constexpr float c2 = -0.7213475204444817f;   // -1 / (2 ln 2)
        constexpr float c3 = 0.48089834696298783f;   //  1 / (3 ln 2)
        constexpr float c4 = -0.36067376022224085f;  // -1 / (4 ln 2)
        constexpr float c5 = 0.28853900817779266f;   //  1 / (5 ln 2)
        constexpr float c6 = -0.24044917348149392f;  // -1 / (6 ln 2)
        return t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, fmaf(t, c6, c5), c4), c3), c2), c1);
    }
    return log2f(y);
}

// Column update after the row sums: warp reduce-scatter of cs, one barrier, then every warp sums
// the per-warp partials of its lanes' columns and updates its copy of g'. With REC, rec_g / rec_cs
// (nc floats each) receive the iteration's g' before the update and its column sums.
template <int NCB, int GPL, bool REC = false>
__device__ __forceinline__ void column_update(float (&cs)[NCB], float (&gm)[GPL], int nc,
                                              float* s_red, const float* s_ib, int par, int lane,
                                              int warp, int W, float* rec_g = nullptr,
                                              float* rec_cs = nullptr) {
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
        if (col < nc) {
            float sum = 0.f;
            for (int ww = 0; ww < W; ++ww) sum += buf[ww * P + col];
            if (REC && warp == 0) {
                rec_g[col] = gm[j];
                rec_cs[col] = sum;
            }
            // log2 b - log2 cs = -log2(cs / b): the argument is near 1, so the log2 and the one
            // rounding of cs / b are accurate to ~1e-7 absolute (two logs of ~log2 |I| each would
            // carry ~5e-7 of rounding into every iteration's potentials)
            gm[j] -= log2_near1(fmaxf(sum * s_ib[col], 1e-37f));
        }
    }
}

}  // namespace fr
