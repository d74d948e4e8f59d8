// fr_p1_k21_batch.cu -- batched-market free-cost kernels for exactly 21 columns.
#include "fr_p1.cuh"

namespace fr {

bool p1_variant_k21_batch(int ld, int threads, P1Variant* out) {
    return p1_k21_with(MkBatch{}, ld, threads, out);
}

}  // namespace fr
