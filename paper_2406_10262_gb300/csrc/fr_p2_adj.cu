// fr_p2_adj.cu -- selection and launch of the unrolled-gradient (adjoint) kernel of the per-item
// parametrisation. Instances: exact 21 columns (fr_p2_adj21.cu), exact 11 and 6 columns
// (fr_p2_adj11.cu) with 8, 16 or 24 rows per thread; padded 8 / 16 / 32 column buckets with 8 rows
// per thread (this file). CTAs have at most 256 threads.
#include "fr_p2_adj.cuh"

namespace fr {

namespace {
constexpr int kAdjMaxThreads = 256;

int adj_ncb(int nc) {
    return nc == 21 || nc == 11 || nc == 6 ? nc : (nc <= 8 ? 8 : (nc <= 16 ? 16 : 32));
}
}  // namespace

bool p2_adj_generic(int ncb, int threads, P2Variant* v) {
    switch (ncb) {
        case 8: p2::p2_make_adj<8, 8, false>(threads, v); return true;
        case 16: p2::p2_make_adj<16, 8, false>(threads, v); return true;
        case 32: p2::p2_make_adj<32, 8, false>(threads, v); return true;
        default: return false;
    }
}

bool p2_select_adj(int nc, int I, P2Variant* v) {
    auto threads_for = [&](int R) { return ((I + R - 1) / R + 31) / 32 * 32; };
    const bool exact = nc == 21 || nc == 11 || nc == 6;
    if (nc < 2 || nc > 32) return false;
    int R = 8;
    if (threads_for(8) > kAdjMaxThreads) {
        if (!exact) return false;
        R = threads_for(16) <= kAdjMaxThreads ? 16 : 24;
        if (threads_for(R) > kAdjMaxThreads) return false;
    }
    const int T = threads_for(R);
    if (nc == 21) return p2_adj_k21(R, T, v);
    if (exact) return p2_adj_k11_k6(nc, R, T, v);
    return p2_adj_generic(adj_ncb(nc), T, v);
}

size_t p2_adj_smem(const P2Variant& v, int nc, int ld, int esz, int ce) {
    return p2::adj_layout(adj_ncb(nc), nc, ld, v.adj_threads / 32, esz, ce, nullptr, nullptr);
}

cudaError_t p2_launch_adj(const P2Variant& v, const P2Args& a, cudaStream_t s) {
    void* args[] = {const_cast<P2Args*>(&a)};
    return cudaLaunchKernel(v.adj, dim3(a.G), dim3(v.adj_threads), args,
                            p2_adj_smem(v, a.nc, a.ld, a.r_bf16 ? 2 : 4, a.ce), s);
}

}  // namespace fr
