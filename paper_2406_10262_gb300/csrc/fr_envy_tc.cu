// fr_envy_tc.cu -- the envy contraction E = R^T V of the Sec. 4.1 metrics on the 5th-generation
// tensor cores (tcgen05), with FP32-level accuracy from three TF32 products.
//
// E_ij = sum_u r(u,i) v_uj. Every FP32 input x is split into two TF32 parts, x = hi + lo with
// hi = tf32(x), lo = tf32(x - hi), and a tile of E accumulates hi_r hi_v + hi_r lo_v + lo_r hi_v in
// FP32 in tensor memory (the dropped lo_r lo_v term is ~2^-22 relative).
//
// Two kernels:
//  - envy_split_kernel writes R and V once as TF32 hi / lo planes, already in the operand layout the
//    tensor cores read from shared memory: one 16 KB block per (128-item tile, 32-consumer stage,
//    part), K-major without swizzle (8-row x 16-byte core matrices, core matrices adjacent in K 128
//    bytes apart, 8-row groups 1024 bytes apart). O(|U| |I|) work.
//  - envy_tc_kernel: a CTA owns a 128 x 256 tile of E (items i x items j) and runs three roles.
//    One producer thread bulk-copies each stage's six blocks (A hi / lo from R's planes of tile i,
//    B hi / lo from V's planes of the two 128-item tiles of j, which land as one 256-row operand;
//    96 KB) into a ring of NS shared buffers. One MMA thread waits for a stage, issues its 12 MMAs
//    (M = 128, N = 256, K = 8; tcgen05.mma.cta_group::1.kind::tf32) and commits them to the stage's
//    "empty" mbarrier, which frees the buffer when they are done. Eight epilogue warps add each
//    completed chunk of 256 consumers (8 stages) from one of two 256-column tensor-memory regions
//    (all 512 columns) to FP32 running sums in registers (tcgen05.ld) while the next chunk
//    accumulates in the other region; restarting the accumulator every 256 consumers keeps the
//    tensor cores' FP32 accumulation within FP32 rounding of an exact sum. The kernel keeps only the
//    row maxima over the tile's valid columns and E_ii where the tile crosses the diagonal: the
//    |I|^2 matrix is never written. The 256-wide tile reads 3/4 of the operand bytes per product
//    of a 128 x 128 tile, from L2 and from shared memory alike.
//
// Every wait is bounded (the context's poll limit). When one expires the CTA records an error
// flag, the other roles give up at their next wait, the producer waits (default bound) for the
// copies it issued and the MMA thread for its last commit, and only then is the tensor memory freed.
#include <cuda_bf16.h>

#include "fr_device.cuh"
#include "fr_internal.h"

namespace fr {

namespace {

constexpr int TM = 128;                       // tile rows (items i), MMA M
constexpr int TN = 256;                       // tile columns (items j), MMA N
constexpr int TP = 128;                       // items per plane tile (A: one, B: TN / TP of them)
constexpr int TK = 32;                        // consumers per stage
constexpr int KSTEP = 8;                      // K of one tf32 MMA (32 bytes per row)
constexpr int OPER_BYTES = TP * TK * 4;       // one plane block (128 items, hi or lo): 16 KB
constexpr int A_BYTES = OPER_BYTES;           // A part of a stage (128 rows)
constexpr int B_BYTES = (TN / TP) * OPER_BYTES;  // B part of a stage (256 rows)
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // A_hi, A_lo, B_hi, B_lo: 96 KB
constexpr int LBO = 128;                      // bytes between K-adjacent core matrices
constexpr int SBO = (TK / 4) * 128;           // bytes between 8-row groups
constexpr int NS = 2;                         // shared stage buffers in the ring
constexpr unsigned kTmemCols = 2 * TN;        // two FP32 accumulator regions of TN columns: 512
constexpr int CHUNK = 8;                      // stages (8 x 32 consumers) per accumulator chunk
constexpr int NEPI = 8;                       // epilogue warps (warps 2 .. 9)
constexpr int NTHREADS = 32 * (2 + NEPI);     // producer warp, MMA warp, epilogue warps
constexpr int ECOLS = TN / 2;                 // columns per epilogue warp
constexpr int kGroupM = 16;                   // row tiles per group of the CTA order

static_assert(TM == 128 && TN % 16 == 0 && TN >= 16 && TN <= 256, "MMA shape");
static_assert(TN % TP == 0 && TM == TP, "operands assembled from 128-item plane blocks");
static_assert(NEPI == 8, "each epilogue warp: one lane quarter, half of the columns");
static_assert(kTmemCols <= 512, "tensor memory columns");

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

// Byte offset of element (row m, k) of a K-major operand part of 32 columns (any number of rows).
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

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for phase `parity` of `bar` that also gives up once another role raised *abort.
__device__ __forceinline__ bool wait_or_abort(unsigned long long* bar, unsigned parity,
                                              unsigned max_polls, volatile int* abort) {
    for (unsigned it = 0; it < max_polls; ++it) {
        unsigned done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (*abort) return false;
    }
    return false;
}

// TF32 planes of an |U| x |I| operand (x = r, or V): for tile t = 0 .. nt-1 (128 items), stage
// s = 0 .. nk-1 (32 consumers) and part p (0 hi, 1 lo), the 16 KB block at ((t nk + s) 2 + p) * 4096
// words holds element (item t 128 + m, consumer s 32 + k) at oper_off(m, k). Entries beyond the
// items or the consumers are 0. One CTA per (t, s); thread (m, g) writes consumers 4g .. 4g+3 of
// row m, one 16-byte vector per part.
__global__ void __launch_bounds__(1024) envy_split_kernel(const void* __restrict__ x, int x_bf16,
                                                          int U, int I, int ld, int nk,
                                                          unsigned* __restrict__ planes) {
    const int t = blockIdx.y, s = blockIdx.x;
    const int m = threadIdx.x % TP, g = threadIdx.x / TP;
    const int i = t * TP + m;
    uint4 hi, lo;
    unsigned* ph = &hi.x;
    unsigned* pl = &lo.x;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int u = s * TK + 4 * g + q;
        const float v = (u < U && i < I) ? rval_tc(x, x_bf16, (size_t)u * ld + i) : 0.f;
        ph[q] = to_tf32(v);
        pl[q] = to_tf32(v - __uint_as_float(ph[q]));
    }
    unsigned char* blk = reinterpret_cast<unsigned char*>(planes + (size_t)(t * nk + s) * 2 * (OPER_BYTES / 4));
    const int o = oper_off(m, 4 * g);
    *reinterpret_cast<uint4*>(blk + o) = hi;
    *reinterpret_cast<uint4*>(blk + OPER_BYTES + o) = lo;
}

// Shared memory: NS stage buffers, then the mbarriers (full / empty per stage, chunk-done / region-
// free per accumulator region), the tensor-memory address and the abort flag.
constexpr int SMEM_BARS = NS * STAGE_BYTES;
constexpr int SMEM_BYTES = SMEM_BARS + (2 * NS + 4) * 8 + 16;

__global__ void __launch_bounds__(NTHREADS, 1) envy_tc_kernel(const unsigned* __restrict__ Rp,
                                                        const unsigned* __restrict__ Vp, int I,
                                                        int ld, int nk, int nt, int ntj,
                                                        float* __restrict__ rmax,
                                                        float* __restrict__ diag, int* err,
                                                        unsigned max_polls) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* stages = smem_raw;
    unsigned long long* full = reinterpret_cast<unsigned long long*>(smem_raw + SMEM_BARS);
    unsigned long long* empty = full + NS;
    unsigned long long* accf = empty + NS;  // chunk accumulated in region r
    unsigned long long* acce = accf + 2;    // region r read by every epilogue warp
    unsigned* tmem_slot = reinterpret_cast<unsigned*>(acce + 2);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // CTA b -> tile (ti, tj): groups of kGroupM row tiles, column tiles in order within a group and
    // row tiles fastest, so the CTAs resident at one time cover a compact block of tiles and reuse
    // each other's operand tiles from L2 instead of streaming all of V once per row of tiles
    const int per_group = kGroupM * ntj, grp = blockIdx.x / per_group, first = grp * kGroupM;
    const int gm = min(nt - first, kGroupM), rem = blockIdx.x - grp * per_group;
    const int ti = first + rem % gm, tj = rem / gm;
    const int i0 = ti * TM, j0 = tj * TN;

    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(full + s, 1);
            mbar_init(empty + s, 1);
        }
        for (int r = 0; r < 2; ++r) {
            mbar_init(accf + r, 1);
            mbar_init(acce + r, NEPI);
        }
        *abort = 0;
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
    const int nch = (nk + CHUNK - 1) / CHUNK;

    // Epilogue warps' running sums: warp w holds the tile rows of its tensor-memory lane quarter,
    // 32 (w % 4) + lane, and the 128 columns 128 ((w - 2) / 4) .. + 127.
    const int q4 = warp & 3, half = (warp - 2) >> 2;
    float sum[ECOLS];
#pragma unroll
    for (int q = 0; q < ECOLS; ++q) sum[q] = 0.f;

    if (warp == 0) {
        if (lane == 0) {  // producer: the stage's six 16 KB blocks into the ring
            const size_t tile_bytes = (size_t)nk * 2 * OPER_BYTES;  // one plane tile, all stages
            const unsigned char* ra = reinterpret_cast<const unsigned char*>(Rp) + (size_t)ti * tile_bytes;
            const unsigned char* vb =
                reinterpret_cast<const unsigned char*>(Vp) + (size_t)tj * (TN / TP) * tile_bytes;
            int last = -1;
            for (int kc = 0; kc < nk; ++kc) {
                const int s = kc % NS;
                if (kc >= NS && !wait_or_abort(empty + s, ((kc / NS) - 1) & 1u, max_polls, abort)) {
                    *abort = 1;
                    break;
                }
                unsigned char* st = stages + s * STAGE_BYTES;
                const size_t kb = (size_t)kc * 2 * OPER_BYTES;
                mbar_arrive_expect_tx(full + s, STAGE_BYTES);
                bulk_g2s(st, ra + kb, OPER_BYTES, full + s);                       // A hi
                bulk_g2s(st + A_BYTES, ra + kb + OPER_BYTES, OPER_BYTES, full + s);  // A lo
#pragma unroll
                for (int h = 0; h < TN / TP; ++h) {  // B hi, B lo: rows h 128 .. of the operand
                    const unsigned char* vt = vb + h * tile_bytes + kb;
                    bulk_g2s(st + 2 * A_BYTES + h * OPER_BYTES, vt, OPER_BYTES, full + s);
                    bulk_g2s(st + 2 * A_BYTES + B_BYTES + h * OPER_BYTES, vt + OPER_BYTES, OPER_BYTES,
                             full + s);
                }
                last = kc;
            }
            // every copy issued here has landed before the CTA can leave (the last fill of each
            // buffer; earlier ones were consumed before the buffer was refilled)
            for (int kc = last - NS + 1 > 0 ? last - NS + 1 : 0; kc <= last; ++kc)
                mbar_wait(full + kc % NS, (kc / NS) & 1u, kDefaultPolls);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            int last = -1;
            for (int kc = 0; kc < nk; ++kc) {
                const int s = kc % NS, c = kc / CHUNK;
                if (kc % CHUNK == 0 && c >= 2 &&
                    !wait_or_abort(acce + (c & 1), ((c >> 1) - 1) & 1u, max_polls, abort)) {
                    *abort = 1;
                    break;
                }
                if (!wait_or_abort(full + s, (kc / NS) & 1u, max_polls, abort)) {
                    *abort = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned base = smem_u32(stages + s * STAGE_BYTES);
                const unsigned dst = tmem + (unsigned)((c & 1) * TN);
                const bool first = kc % CHUNK == 0;
#pragma unroll
                for (int ks = 0; ks < TK / KSTEP; ++ks) {
                    const unsigned koff = (unsigned)(ks * 2 * LBO);  // two core matrices per K step
                    const unsigned long long ah = smem_desc(base + koff);
                    const unsigned long long al = smem_desc(base + A_BYTES + koff);
                    const unsigned long long bh = smem_desc(base + 2 * A_BYTES + koff);
                    const unsigned long long bl = smem_desc(base + 2 * A_BYTES + B_BYTES + koff);
                    mma_tf32(dst, ah, bh, (first && ks == 0) ? 0u : 1u);
                    mma_tf32(dst, ah, bl, 1u);
                    mma_tf32(dst, al, bh, 1u);
                }
                mma_commit(empty + s);  // the buffer is free once these MMAs are done
                if (kc % CHUNK == CHUNK - 1 || kc == nk - 1) mma_commit(accf + (c & 1));
                last = kc;
            }
            // no MMA of this CTA is still running when it frees the tensor memory
            if (last >= 0) mbar_wait(empty + last % NS, (last / NS) & 1u, kDefaultPolls);
        }
    } else {  // epilogue: chunk c of region c & 1 into the running sums, then free the region
        for (int c = 0; c < nch; ++c) {
            const bool w = wait_or_abort(accf + (c & 1), (c >> 1) & 1u, max_polls, abort);
            if (!__all_sync(FULL, w)) {
                *abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int h = 0; h < ECOLS / 32; ++h) {
                unsigned v[32];
                const unsigned taddr = tmem + ((unsigned)(q4 * 32) << 16) +
                                       (unsigned)((c & 1) * TN + half * ECOLS + h * 32);
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
                for (int q = 0; q < 32; ++q) sum[h * 32 + q] += __uint_as_float(v[q]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(acce + (c & 1));
        }
    }

    __syncthreads();  // every role is done (or gave up) and drained its own asynchronous work
    const bool good = *abort == 0;
    float* red = reinterpret_cast<float*>(stages);  // the stage buffers are idle now
    if (!good) {
        if (tid == 0) atomicOr(err, 4);
    } else if (warp >= 2) {
        // row maxima over the tile's valid columns (this warp's 128), and E_ii where column j = i
        // lies among them
        const int row = q4 * 32 + lane, i = i0 + row, jw = j0 + half * ECOLS;
        float m = -INFINITY, d = 0.f;
#pragma unroll
        for (int q = 0; q < ECOLS; ++q) {
            if (jw + q < I) m = fmaxf(m, sum[q]);
            if (jw + q == i) d = sum[q];
        }
        if (i >= jw && i < jw + ECOLS && i < I) diag[i] = d;
        red[half * TM + row] = m;
    }
    __syncthreads();
    if (good && warp >= 2 && half == 0) {
        const int row = q4 * 32 + lane, i = i0 + row;
        if (i < I) rmax[(size_t)tj * ld + i] = fmaxf(red[row], red[TM + row]);
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
int envy_tc_col_tiles(int I) { return (I + TN - 1) / TN; }
size_t envy_tc_smem() { return SMEM_BYTES; }
size_t envy_tc_plane_bytes(int U, int I) {
    // R: one plane tile per 128 items; V: TN / TP per 256-item column tile (zero past the items)
    const size_t nt = (size_t)envy_tc_tiles(I), ntv = (size_t)envy_tc_col_tiles(I) * (TN / TP);
    const size_t nk = (size_t)(U + TK - 1) / TK;
    return (nt + ntv) * nk * 2 * OPER_BYTES;  // hi and lo
}

cudaError_t launch_envy_tc(const void* r, int r_bf16, const float* V, int U, int I, int ld,
                           float* rmax, float* diag, int* err, unsigned max_polls, void* planes,
                           cudaStream_t s) {
    const int nt = envy_tc_tiles(I), ntj = envy_tc_col_tiles(I), nk = (U + TK - 1) / TK;
    unsigned* Rp = static_cast<unsigned*>(planes);
    unsigned* Vp = Rp + (size_t)nt * nk * 2 * (OPER_BYTES / 4);
    envy_split_kernel<<<dim3(nk, nt), 1024, 0, s>>>(r, r_bf16, U, I, ld, nk, Rp);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    envy_split_kernel<<<dim3(nk, ntj * (TN / TP)), 1024, 0, s>>>(V, 0, U, I, ld, nk, Vp);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = raise_smem_limit((const void*)envy_tc_kernel, envy_tc_smem())) != cudaSuccess) return e;
    envy_tc_kernel<<<nt * ntj, NTHREADS, envy_tc_smem(), s>>>(Rp, Vp, I, ld, nk, nt, ntj, rmax,
                                                             diag, err, max_polls);
    return cudaGetLastError();
}

}  // namespace fr
