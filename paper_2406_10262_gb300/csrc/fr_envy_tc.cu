// fr_envy_tc.cu -- the envy contraction E = R^T V of the Sec. 4.1 metrics on the 5th-generation
// tensor cores (tcgen05), with FP32-level accuracy from three TF32 products.
//
// E_ij = sum_u r(u,i) v_uj. A CTA owns a 128 x 128 tile of E (items i x items j); the contraction
// index u (consumers) is streamed 32 at a time. Every FP32 input x is split into two TF32 parts,
// x = hi + lo with hi = tf32(x), lo = tf32(x - hi), and the tile accumulates
//   hi_r hi_v + hi_r lo_v + lo_r hi_v
// in FP32 in tensor memory (the dropped lo_r lo_v term is ~2^-22 relative): 12 MMAs of
// M = 128, N = 128, K = 8 per 32 consumers, issued by one thread (tcgen05.mma.cta_group::1.
// kind::tf32) and tracked by an mbarrier through tcgen05.commit. Operands live in shared memory in
// the K-major, no-swizzle canonical layout: 8-row x 16-byte core matrices, core matrices adjacent
// in K 128 bytes apart (leading byte offset), 8-row groups 1024 bytes apart (stride byte offset).
// The CTA's 512 threads stage the next 32 consumers (two shared buffers, operands loaded into
// registers two stages ahead) while the tensor cores work on the current ones. The epilogue reads the accumulator rows back from tensor memory (tcgen05.ld,
// 32 lanes per warp) and keeps only the row maxima over the tile's valid columns and, on diagonal
// tiles, E_ii: the |I|^2 matrix is never written.
//
// Every wait is bounded; on expiry the kernel records an error flag, waits (bounded) for its own
// MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include "fr_device.cuh"
#include "fr_internal.h"

namespace fr {

namespace {

constexpr int TM = 128;                       // tile rows (items i), MMA M
constexpr int TN = 128;                       // tile columns (items j), MMA N
constexpr int TK = 32;                        // consumers per stage
constexpr int KSTEP = 8;                      // K of one tf32 MMA (32 bytes per row)
constexpr int OPER_BYTES = TM * TK * 4;       // one operand part (hi or lo) of one stage: 16 KB
constexpr int STAGE_BYTES = 4 * OPER_BYTES;   // A_hi, A_lo, B_hi, B_lo
constexpr int LBO = 128;                      // bytes between K-adjacent core matrices
constexpr int SBO = (TK / 4) * 128;           // bytes between 8-row groups
constexpr unsigned kTmemCols = 2 * TN;        // two FP32 accumulator regions of TN columns
constexpr int CHUNK = 8;                      // stages (8 x 32 consumers) per accumulator chunk
constexpr int NTHREADS = 512;                 // staging threads (warps 0-3 also run the epilogue)
constexpr int KGROUPS = NTHREADS / TM;        // groups of 4 consumers per stage per thread row

static_assert(TM == 128 && TN % 16 == 0 && TN >= 16 && TN <= 256, "MMA shape");
static_assert(TN == TM, "square tiles (diagonal capture)");

__device__ __forceinline__ float rval_tc(const void* r, int bf16, size_t o) {
    return bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(r)[o])
                : static_cast<const float*>(r)[o];
}

// x rounded to TF32 (10 explicit mantissa bits), to nearest with ties away from zero, in two integer
// operations: add half a TF32 unit in the last place to the magnitude bits, then clear the 13
// dropped bits (a carry into the exponent is the correct rounding up to the next binade).
__device__ __forceinline__ unsigned to_tf32(float x) {
    return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

// Byte offset of element (row m, k) of a 128 x 32 K-major operand part.
__host__ __device__ constexpr int oper_off(int m, int k) {
    return (m / 8) * SBO + (k / 4) * LBO + (m % 8) * 16 + (k % 4) * 4;
}

__device__ __forceinline__ unsigned long long smem_desc(unsigned addr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((addr >> 4) & 0x3FFF);
    d |= (unsigned long long)((LBO >> 4) & 0x3FFF) << 16;
    d |= (unsigned long long)((SBO >> 4) & 0x3FFF) << 32;
    d |= 1ull << 46;  // descriptor version of this tensor-core generation; no swizzle (bits 61-63 = 0)
    return d;
}

// kind::tf32 instruction descriptor: D = F32, A = B = TF32, both K-major, M = 128, N = TN.
constexpr unsigned kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(TN >> 3) << 17) |
                            ((unsigned)(TM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(unsigned tmem_d, unsigned long long a, unsigned long long b,
                                         unsigned accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(unsigned long long* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// One stage = 32 consumers of the tile: A[m][k] = r(u0 + k, i0 + m), B[n][k] = v(u0 + k, j0 + n).
// Thread t owns row t % 128 of both operands and the groups of 4 consumers g0 + KGROUPS q,
// g0 = t / 128. load_stage reads them into registers (issued two stages ahead, so the global-memory
// latency overlaps the tensor cores' work); store_stage splits each value into TF32 hi and lo parts
// and writes one 16-byte vector per group and part.
constexpr int QG = TK / 4 / KGROUPS;  // groups per thread per stage

struct StageRegs {
    float r[QG][4], v[QG][4];
};

__device__ __forceinline__ void load_stage(StageRegs& R, const void* r, int r_bf16, const float* V,
                                           int U, int ld, int i0, int j0, int u0) {
    const int t = threadIdx.x % TM, g0 = threadIdx.x / TM;
    const int i = i0 + t, j = j0 + t;
#pragma unroll
    for (int q2 = 0; q2 < QG; ++q2) {
        const int k4 = 4 * (g0 + KGROUPS * q2);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int u = u0 + k4 + q;
            R.r[q2][q] = (u < U && i < ld) ? rval_tc(r, r_bf16, (size_t)u * ld + i) : 0.f;
            R.v[q2][q] = (u < U && j < ld) ? V[(size_t)u * ld + j] : 0.f;
        }
    }
}

__device__ __forceinline__ void store_stage(unsigned char* st, const StageRegs& R) {
    const int t = threadIdx.x % TM, g0 = threadIdx.x / TM;
#pragma unroll
    for (int q2 = 0; q2 < QG; ++q2) {
        const int k4 = 4 * (g0 + KGROUPS * q2);
        uint4 rh, rl, vh, vl;
        unsigned* prh = &rh.x; unsigned* prl = &rl.x; unsigned* pvh = &vh.x; unsigned* pvl = &vl.x;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            prh[q] = to_tf32(R.r[q2][q]);
            prl[q] = to_tf32(R.r[q2][q] - __uint_as_float(prh[q]));
            pvh[q] = to_tf32(R.v[q2][q]);
            pvl[q] = to_tf32(R.v[q2][q] - __uint_as_float(pvh[q]));
        }
        const int o = oper_off(t, k4);
        *reinterpret_cast<uint4*>(st + 0 * OPER_BYTES + o) = rh;
        *reinterpret_cast<uint4*>(st + 1 * OPER_BYTES + o) = rl;
        *reinterpret_cast<uint4*>(st + 2 * OPER_BYTES + o) = vh;
        *reinterpret_cast<uint4*>(st + 3 * OPER_BYTES + o) = vl;
    }
}

__global__ void __launch_bounds__(NTHREADS, 1) envy_tc_kernel(const void* __restrict__ r, int r_bf16,
                                                        const float* __restrict__ V, int U, int I,
                                                        int ld, float* __restrict__ rmax,
                                                        float* __restrict__ diag, int* err,
                                                        unsigned max_polls) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* stages = smem_raw;                                    // 2 x STAGE_BYTES
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw + 2 * STAGE_BYTES);
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(bar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = blockIdx.y * TM, j0 = blockIdx.x * TN;

    if (tid == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = *tmem_slot;

    // Running sums of the tile in registers: warp w holds the tile rows of its tensor-memory lane
    // quarter, 32 (w % 4) + lane, and the 32 columns 32 (w / 4) .. + 31.
    const int q4 = warp & 3, cslice = warp >> 2;
    float sum[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) sum[q] = 0.f;
    auto read_chunk = [&](int c) {  // adds chunk c's accumulator (region c & 1) to the sums
        unsigned v[32];
        const unsigned taddr = tmem + ((unsigned)(q4 * 32) << 16) + (unsigned)((c & 1) * TN + cslice * 32);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
            "%10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, "
            "%26, %27, %28, %29, %30, %31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
              "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
              "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]),
              "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
              "=r"(v[30]), "=r"(v[31])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int q = 0; q < 32; ++q) sum[q] += __uint_as_float(v[q]);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    };

    const int nk = (U + TK - 1) / TK;
    const int nch = (nk + CHUNK - 1) / CHUNK;
    bool ok = true;
    int issued = -1;  // last stage whose MMAs were committed
    int nread = 0;    // chunks added to the running sums (in order)
    StageRegs regs;
    load_stage(regs, r, r_bf16, V, U, ld, i0, j0, 0);
    for (int kc = 0; kc < nk; ++kc) {
        const int st = kc & 1;
        unsigned char* sbuf = stages + st * STAGE_BYTES;
        if (kc >= 2 && ok) {  // the MMAs that read this buffer two stages ago are done
            if (!mbar_wait(bar + st, ((kc - 2) >> 1) & 1u, max_polls)) ok = false;
        }
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        // the chunk that ended with stage kc - 2 is complete (waited for just above): add it
        // before chunk kc / CHUNK + 1 reuses its region
        if (kc % CHUNK == 1 && kc > CHUNK) read_chunk(nread++);
        store_stage(sbuf, regs);
        if (kc + 1 < nk) load_stage(regs, r, r_bf16, V, U, ld, i0, j0, (kc + 1) * TK);
        fence_proxy_async_smem();  // generic-proxy stores -> the tensor cores' (async proxy) reads
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned base = smem_u32(sbuf);
            const unsigned dst = tmem + (unsigned)(((kc / CHUNK) & 1) * TN);
            const bool first = kc % CHUNK == 0;
#pragma unroll
            for (int ks = 0; ks < TK / KSTEP; ++ks) {
                const unsigned koff = (unsigned)(ks * 2 * LBO);  // two core matrices per K step
                const unsigned long long ah = smem_desc(base + 0 * OPER_BYTES + koff);
                const unsigned long long al = smem_desc(base + 1 * OPER_BYTES + koff);
                const unsigned long long bh = smem_desc(base + 2 * OPER_BYTES + koff);
                const unsigned long long bl = smem_desc(base + 3 * OPER_BYTES + koff);
                mma_tf32(dst, ah, bh, (first && ks == 0) ? 0u : 1u);
                mma_tf32(dst, ah, bl, 1u);
                mma_tf32(dst, al, bh, 1u);
            }
            mma_commit(bar + st);
        }
        issued = kc;
    }
    // all MMAs complete: the last commit tracks every earlier one of the issuing thread. If this
    // wait (or an earlier one) expired, the CTA still waits, with the default bound, for its own
    // MMAs before it frees the tensor memory and leaves.
    if (issued >= 0 && !mbar_wait(bar + (issued & 1), (issued >> 1) & 1u, ok ? max_polls : 0u))
        ok = false;
    if (issued >= 0 && !__syncthreads_and(ok))
        mbar_wait(bar + (issued & 1), (issued >> 1) & 1u, kDefaultPolls);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!__syncthreads_and(ok)) {
        if (tid == 0) atomicOr(err, 4);
    } else {
        while (nread < nch) read_chunk(nread++);  // the last one or two chunks
        // row maxima over the tile's valid columns: each warp over its 32 columns, then the four
        // column slices of a row combined through shared memory (the stage buffers are idle now)
        const int row = q4 * 32 + lane, i = i0 + row;
        float m = -INFINITY, d = 0.f;
#pragma unroll
        for (int q = 0; q < 32; ++q) {
            if (j0 + cslice * 32 + q < I) m = fmaxf(m, sum[q]);
            if (q == lane) d = sum[q];
        }
        if (i0 == j0 && cslice == q4 && i < I) diag[i] = d;  // column j = i sits in this slice
        float* red = reinterpret_cast<float*>(stages);
        red[cslice * TM + row] = m;
        __syncthreads();
        if (warp < TM / 32 && i < I) {
            float mm = red[row];
#pragma unroll
            for (int sl = 1; sl < TN / 32; ++sl) mm = fmaxf(mm, red[sl * TM + row]);
            rmax[(size_t)blockIdx.x * ld + i] = mm;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
}

}  // namespace

int envy_tc_tiles(int I) { return (I + TM - 1) / TM; }
size_t envy_tc_smem() { return 2 * STAGE_BYTES + 64; }

cudaError_t launch_envy_tc(const void* r, int r_bf16, const float* V, int U, int I, int ld,
                           float* rmax, float* diag, int* err, unsigned max_polls,
                           cudaStream_t s) {
    const int nt = envy_tc_tiles(I);
    cudaError_t e = raise_smem_limit((const void*)envy_tc_kernel, envy_tc_smem());
    if (e != cudaSuccess) return e;
    envy_tc_kernel<<<dim3(nt, nt), NTHREADS, envy_tc_smem(), s>>>(r, r_bf16, V, U, I, ld, rmax, diag,
                                                                 err, max_polls);
    return cudaGetLastError();
}

}  // namespace fr
