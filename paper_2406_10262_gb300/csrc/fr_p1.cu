// fr_p1.cu -- variant table and launch of the free-cost kernels (fr_p1.cuh).
#include "fr_p1.cuh"

namespace fr {

bool p1_variant_k21(int ld, int threads, P1Variant* out);  // fr_p1_k21.cu

size_t p1_smem_bytes(const P1Variant& v, int mode, int nc, int ld) {
    return smem_layout(v.ncb, nc, ld, v.threads / 32, mode, v.tile_stride, nullptr, nullptr);
}

bool p1_select(int nc, int I, P1Variant* out) {
    return p1_select_with(MkPlain{}, nc, I, out, p1_variant_k21);
}

cudaError_t p1_launch(const P1Variant& v, int mode, const P1Args& a, cudaStream_t s) {
    const size_t smem = p1_smem_bytes(v, mode, a.nc, a.ld);
    void* args[] = {const_cast<P1Args*>(&a)};
    // the unrolled gradient's solves record every iteration (its own compiled kernel)
    const void* fn = (mode == MODE_SWEEP && a.gall) ? v.fn_rec : v.fn[mode];
    return cudaLaunchKernel(fn, dim3(a.G), dim3(v.threads), args, smem, s);
}

}  // namespace fr
