// fr_noalloc.cu -- fr_nsw_eval_noalloc: the Sinkhorn solve and impact reduction of the free-cost
// path for callers that cannot allocate device memory.
//
// Every piece of scratch memory the kernels need -- per-CTA impact partials, the reduction's
// per-block sums, the step-state record, the column potentials and the padded exposure -- lives in
// one file-scope static __device__ array of kScratchBytes bytes. The CUDA runtime reserves it on
// every device that loads this library, for the life of the process; the entry point itself calls
// no cudaMalloc/cudaFree and no allocating library routine.
//
// Host code must not take the address of g_scratch directly: on the host the symbol is only a
// stand-in. The device address is looked up once per device with cudaGetSymbolAddress (with that
// device current) on the first call made on that device, and cached.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "fairrank.h"
#include "fr_internal.h"

namespace fr {
void set_thread_error(const char* msg);  // fr_api.cu: message returned by fr_last_error(NULL)

namespace {

constexpr size_t kScratchBytes = size_t(8) << 20;  // 8 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

struct ExposurePack {
    float e[64];
    float invb[64];
};

// Writes the padded exposure / log2 marginals and clears the step-state record (its reduction
// ticket must start at zero on every call, since the array keeps the previous call's contents).
__global__ void noalloc_prepare(ExposurePack p, int nc, float* e, float* ib, DevState* st) {
    const int k = threadIdx.x;
    if (k < nc) {
        e[k] = p.e[k];
        ib[k] = p.invb[k];
    }
    if (k == 0) {
        DevState z{};
        z.thresh = -1.0;
        *st = z;
    }
}

__global__ void noalloc_finish(const DevState* st, double* out) {
    out[0] = st->F;
    out[1] = st->utility;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace
}  // namespace fr

using namespace fr;

extern "C" fr_status fr_nsw_eval_noalloc(const float* C, const float* r, int64_t ld,
                                         const double* e, int32_t n_users, int32_t n_items,
                                         int32_t n_slots, double epsilon, int32_t sinkhorn_iters,
                                         double* imp_out, double* nsw_util_out, void* stream) {
    auto bad = [](fr_status st, const char* msg) {
        set_thread_error(msg);
        return st;
    };
    // A failed CUDA call: the message names the step and the runtime's error string; the
    // runtime's last-error slot is cleared so that the caller's next error check does not see it.
    auto cuda_fail = [](const char* what, cudaError_t err) {
        char buf[256];
        std::snprintf(buf, sizeof buf, "fr_nsw_eval_noalloc: %s: %s", what, cudaGetErrorString(err));
        set_thread_error(buf);
        (void)cudaGetLastError();
        return FR_ECUDA;
    };
    if (!C || !r || !e || !imp_out || !nsw_util_out)
        return bad(FR_EINVAL, "fr_nsw_eval_noalloc: NULL pointer argument");
    if (n_users < 1 || n_items < 1 || n_slots < 1 || n_slots > n_items)
        return bad(FR_EINVAL, "fr_nsw_eval_noalloc: need n_users >= 1 and 1 <= n_slots <= n_items");
    if (!(epsilon > 0.0) || !std::isfinite(epsilon) || sinkhorn_iters < 1)
        return bad(FR_EINVAL, "fr_nsw_eval_noalloc: need epsilon > 0 and sinkhorn_iters >= 1");
    if (ld < n_items || ld % 8 != 0 || ld > (int64_t)1 << 30)
        return bad(FR_EINVAL, "fr_nsw_eval_noalloc: ld must be a multiple of 8 and >= n_items");
    if (reinterpret_cast<uintptr_t>(C) % 16 || reinterpret_cast<uintptr_t>(r) % 16)
        return bad(FR_EINVAL, "fr_nsw_eval_noalloc: C and r must be 16-byte aligned");
    const int nc = fr_num_cols(n_items, n_slots);
    if (nc > 64) return bad(FR_EUNSUPPORTED, "fr_nsw_eval_noalloc: at most 64 columns");
    ExposurePack pack{};
    for (int k = 0; k < n_slots; ++k) {
        if (!(e[k] > 0.0) || !std::isfinite(e[k]))
            return bad(FR_EINVAL, "fr_nsw_eval_noalloc: exposure must be positive and finite");
        pack.e[k] = (float)e[k];
    }
    for (int k = 0; k < nc; ++k) pack.invb[k] = 1.f;  // 1 / b_k
    if (nc > n_slots) pack.invb[n_slots] = (float)(1.0 / (double)(n_items - n_slots));
    P1Variant var;
    if (!p1_select(nc, n_items, &var))
        return bad(FR_EUNSUPPORTED,
                   "fr_nsw_eval_noalloc: n_cols / n_items outside the compiled kernel variants");

    int dev = 0, sms = 0, occ = 0, max_optin = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce != cudaSuccess) return cuda_fail("cudaGetDevice", ce);
    if (dev < 0 || dev >= kMaxDevices)
        return bad(FR_EUNSUPPORTED, "fr_nsw_eval_noalloc: device ordinal above 63");
    {
        // once per device, with that device current: the device address of the static array
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            ce = cudaGetSymbolAddress(&p, g_scratch);
            if (ce != cudaSuccess) return cuda_fail("cudaGetSymbolAddress of the scratch array", ce);
            if (!p) return bad(FR_ECUDA, "fr_nsw_eval_noalloc: scratch array has no device address");
            g_scratch_ptr[dev] = p;
        }
    }
    unsigned char* base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    if ((ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail("cudaDeviceGetAttribute(multiprocessor count)", ce);
    if ((ce = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
        cudaSuccess)
        return cuda_fail("cudaDeviceGetAttribute(shared memory per block)", ce);
    // The kernel's dynamic shared memory grows with ld (the staged cost tile); above the 48 KB
    // default its limit must be raised, which a context of the same variant may or may not have
    // done already in this process. Raising it allocates nothing.
    const size_t smem = p1_smem_bytes(var, MODE_SWEEP, nc, (int)ld);
    if (smem > (size_t)max_optin) {
        char buf[192];
        std::snprintf(buf, sizeof buf,
                      "fr_nsw_eval_noalloc: the cost tile needs %zu bytes of shared memory per "
                      "block (device limit %d): reduce ld or n_items",
                      smem, max_optin);
        return bad(FR_EUNSUPPORTED, buf);
    }
    if ((ce = raise_smem_limit(var.fn[MODE_SWEEP], smem)) != cudaSuccess)
        return cuda_fail("raising the kernel's shared-memory limit", ce);
    ce = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, var.fn[MODE_SWEEP], var.threads, smem);
    if (ce != cudaSuccess) return cuda_fail("cudaOccupancyMaxActiveBlocksPerMultiprocessor", ce);
    if (occ < 1)
        return bad(FR_EUNSUPPORTED, "fr_nsw_eval_noalloc: the kernel variant cannot be resident");

    // scratch layout: state | e | invb | omega | blk | gn2_part | gL | gP | part
    const int nblk = reduce_blocks(n_items);
    const size_t fixed = align256(sizeof(DevState)) + 2 * align256(sizeof(float) * 64) +
                         align256(sizeof(float) * ld) + align256(sizeof(double) * 2 * nblk) +
                         2 * align256(sizeof(float) * (size_t)n_users * nc);
    const size_t part_row = sizeof(float) * (size_t)ld;
    int G = std::min(n_users, occ * sms);
    const size_t room = kScratchBytes > fixed ? kScratchBytes - fixed : 0;
    // gn2_part takes G doubles ahead of the partials
    while (G > 0 && align256(sizeof(double) * G) + (size_t)G * part_row > room) --G;
    if (G < 1)  // problem larger than the static scratch
        return bad(FR_EUNSUPPORTED,
                   "fr_nsw_eval_noalloc: 8 MiB static scratch too small: needs "
                   "2*n_users*n_cols + n_items (+ one partial row of ld) floats");

    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base + off;
        off += align256(bytes);
        return p;
    };
    DevState* st = reinterpret_cast<DevState*>(take(sizeof(DevState)));
    float* ed = reinterpret_cast<float*>(take(sizeof(float) * 64));
    float* ib = reinterpret_cast<float*>(take(sizeof(float) * 64));
    float* omega = reinterpret_cast<float*>(take(sizeof(float) * ld));
    double* blk = reinterpret_cast<double*>(take(sizeof(double) * 2 * nblk));
    double* gn2 = reinterpret_cast<double*>(take(sizeof(double) * G));
    float* gL = reinterpret_cast<float*>(take(sizeof(float) * (size_t)n_users * nc));
    float* gP = reinterpret_cast<float*>(take(sizeof(float) * (size_t)n_users * nc));
    float* part = reinterpret_cast<float*>(take((size_t)G * part_row));
    if (off > kScratchBytes)
        return bad(FR_EUNSUPPORTED, "fr_nsw_eval_noalloc: 8 MiB static scratch too small");

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    {
        int nc_arg = nc;
        void* args[] = {&pack, &nc_arg, &ed, &ib, &st};
        ce = cudaLaunchKernel((const void*)noalloc_prepare, dim3(1), dim3(64), args, 0, s);
        if (ce != cudaSuccess) return cuda_fail("launch of the set-up kernel", ce);
    }

    P1Args a{};
    a.U = n_users; a.I = n_items; a.K = n_slots; a.nc = nc; a.ld = (int)ld;
    a.L = sinkhorn_iters; a.G = G;
    a.C = const_cast<float*>(C);
    a.gL = gL; a.gP = gP; a.r = r; a.e = ed; a.invb = ib; a.omega = omega;
    a.part = part; a.gn2_part = gn2; a.st = st;
    a.inv_eps_ln2 = (float)(1.0 / (epsilon * std::log(2.0)));
    a.inv_eps = (float)(1.0 / epsilon);
    a.warm = 0;  // cold start: the first solve begins from zero column potentials
    a.max_polls = kDefaultPolls;
    if ((ce = p1_launch(var, MODE_SWEEP, a, s)) != cudaSuccess)
        return cuda_fail("launch of the Sinkhorn kernel", ce);

    ReduceArgs ra{};
    ra.I = n_items; ra.ld = (int)ld; ra.G = G; ra.U = n_users;
    ra.part = part; ra.gn2_part = gn2; ra.imp = imp_out; ra.omega = omega; ra.blk = blk; ra.st = st;
    ra.F_hist = nullptr; ra.gn_hist = nullptr; ra.hist_cap = 0; ra.after_update = 0;
    ra.Ggn = 0;
    if ((ce = reduce_launch(ra, s)) != cudaSuccess)
        return cuda_fail("launch of the impact reduction", ce);
    {
        const DevState* stc = st;
        void* args[] = {&stc, &nsw_util_out};
        ce = cudaLaunchKernel((const void*)noalloc_finish, dim3(1), dim3(1), args, 0, s);
        if (ce != cudaSuccess) return cuda_fail("launch of the result kernel", ce);
    }
    return FR_OK;
}
