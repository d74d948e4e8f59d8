// fr_p1_adj.cu -- variant table and launch of the free-cost unrolled-gradient kernel
// (fr_p1_adj.cuh).
#include "fr_p1_adj.cuh"

namespace fr {
namespace {

template <int NCB, int R, bool EXACT>
P1AdjVariant make_adj(int threads) {
    P1AdjVariant v;
    v.ncb = NCB;
    v.rows = R;
    v.exact = EXACT;
    v.threads = threads;
    v.fn[p1adj::ADJ_GRAD] = (const void*)p1adj::p1_adj_kernel<NCB, R, EXACT, p1adj::ADJ_GRAD>;
    v.fn[p1adj::ADJ_STEP] = (const void*)p1adj::p1_adj_kernel<NCB, R, EXACT, p1adj::ADJ_STEP>;
    return v;
}

}  // namespace

// A thread holds R rows' dL/dc (R x NCB registers): 4 rows up to 16 columns (at most 1024 items),
// 2 rows for 21 and up to 32 columns (512 items); CTAs of at most 256 threads.
bool p1_select_adj(int nc, int I, P1AdjVariant* out) {
    auto threads_for = [&](int R) {
        const int t = (I + R - 1) / R;
        return (t + 31) / 32 * 32;
    };
    if (nc == 11 && threads_for(4) <= 256)
        *out = make_adj<11, 4, true>(threads_for(4));
    else if (nc == 21 && threads_for(2) <= 256)
        *out = make_adj<21, 2, true>(threads_for(2));
    else if (nc <= 8 && threads_for(4) <= 256)
        *out = make_adj<8, 4, false>(threads_for(4));
    else if (nc <= 16 && threads_for(4) <= 256)
        *out = make_adj<16, 4, false>(threads_for(4));
    else if (nc <= 32 && threads_for(2) <= 256)
        *out = make_adj<32, 2, false>(threads_for(2));
    else
        return false;
    return true;
}

size_t p1_adj_smem(const P1AdjVariant& v, int nc, int ld, int ce, int nck) {
    return p1adj::layout(v.ncb, nc, ld, v.threads / 32, ce, nck, nullptr, nullptr);
}

cudaError_t p1_launch_adj(const P1AdjVariant& v, int mode, const P1Args& a, int G, cudaStream_t s) {
    const size_t smem = p1_adj_smem(v, a.nc, a.ld, a.ce, a.nck);
    void* args[] = {const_cast<P1Args*>(&a)};
    return cudaLaunchKernel(v.fn[mode], dim3(G), dim3(v.threads), args, smem, s);
}

}  // namespace fr
