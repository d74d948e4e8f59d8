// fr_p1_batch.cu -- batched-market forms of the free-cost kernels (p1_batch_kernel): the variant
// table and launch.
#include "fr_p1.cuh"

namespace fr {

bool p1_variant_k21_batch(int ld, int threads, P1Variant* out);  // fr_p1_k21_batch.cu

bool p1_select_batch(int nc, int I, P1Variant* out) {
    return p1_select_with(MkBatch{}, nc, I, out, p1_variant_k21_batch);
}

// MODE_SWEEP and MODE_UPDATE_SWEEP take the same layout size rules as the single-market kernels;
// every market of a launch uses the layout at ld_max with the full column count.
size_t p1_smem_bytes_batch(const P1Variant& v, int mode, int ld_max) {
    return smem_layout(v.ncb, v.ncb, ld_max, v.threads / 32, mode, v.tile_stride, nullptr, nullptr);
}

cudaError_t p1_launch_batch(const P1Variant& v, int mode, const P1Batch& bt, int G, cudaStream_t s) {
    if (G <= 0 || bt.n_chunks <= 0) return cudaSuccess;
    const size_t smem = p1_smem_bytes_batch(v, mode, bt.ld_max);
    void* args[] = {const_cast<P1Batch*>(&bt)};
    return cudaLaunchKernel(v.fb[mode == MODE_UPDATE_SWEEP ? 1 : 0], dim3(G), dim3(v.threads), args,
                            smem, s);
}

}  // namespace fr
