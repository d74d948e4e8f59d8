// fr_p1.cu -- variant table and launch of the free-cost kernels (fr_p1.cuh).
#include "fr_p1.cuh"

namespace fr {

bool p1_variant_k21(int ld, int threads, P1Variant* out);  // fr_p1_k21.cu

size_t p1_smem_bytes(const P1Variant& v, int mode, int nc, int ld) {
    return smem_layout(v.ncb, nc, ld, v.threads / 32, mode, v.tile_stride, nullptr, nullptr);
}

// Compiled variants: exact column counts for the hot shapes, padded buckets for the rest.
bool p1_select(int nc, int I, P1Variant* out) {
    // CTA size: one thread per R items, at most 512 threads (the kernels' launch bound)
    auto threads_for = [&](int R) {
        int t = (I + R - 1) / R;
        return (t + 31) / 32 * 32;
    };
    P1Variant v;
    // 11 columns: costs in registers up to 768 items; beyond that the tile sweep (eight rows per
    // thread, costs read from the resident tile at a compile-time column stride of 1024, 2048 or
    // 4096 floats), up to 4096 items. Measured fused steps: 2000 x 1000 0.485 vs 0.506 ms,
    // 2000 x 2000 0.977 vs 1.126 ms, 250 x 2000 0.148 vs 0.174 ms for the tile sweep; at 250 and
    // 500 items a 1024-float stride leaves one-warp CTAs four to an SM and the tile sweep runs
    // at half the register sweep's speed.
    const int ld = (I + 7) / 8 * 8;
    if (nc == 11 && ld <= 768 && threads_for(4) <= 512) {
        v = make_variant<11, 4, true>(threads_for(4));
    } else if (nc == 11 && threads_for(8) <= 512) {
        if (ld <= 1024)
            v = make_variant<11, 8, true, 1024>(threads_for(8));
        else if (ld <= 2048)
            v = make_variant<11, 8, true, 2048>(threads_for(8));
        else
            v = make_variant<11, 8, true, 4096>(threads_for(8));
    } else if (nc == 21 && threads_for(8) <= 256 && p1_variant_k21(ld, threads_for(8), &v)) {
        // 21 columns: the tile sweep (exact, eight rows per thread, at most 256 threads) up to
        // 2048 items
    } else if (nc == 50 && threads_for(1) <= 512) {
        v = make_variant<50, 1, true>(threads_for(1));
    } else if (nc <= 8 && threads_for(4) <= 512) {
        v = make_variant<8, 4, false>(threads_for(4));
    } else if (nc <= 16 && threads_for(4) <= 512) {
        v = make_variant<16, 4, false>(threads_for(4));
    } else if (nc <= 32 && threads_for(2) <= 512) {
        v = make_variant<32, 2, false>(threads_for(2));
    } else if (nc <= 64 && threads_for(1) <= 512) {
        v = make_variant<64, 1, false>(threads_for(1));
    } else {
        return false;
    }
    *out = v;
    return true;
}

cudaError_t p1_launch(const P1Variant& v, int mode, const P1Args& a, cudaStream_t s) {
    const size_t smem = p1_smem_bytes(v, mode, a.nc, a.ld);
    void* args[] = {const_cast<P1Args*>(&a)};
    return cudaLaunchKernel(v.fn[mode], dim3(a.G), dim3(v.threads), args, smem, s);
}

}  // namespace fr
