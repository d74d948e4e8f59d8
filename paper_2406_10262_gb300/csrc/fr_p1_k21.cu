// fr_p1_k21.cu -- free-cost kernels compiled for exactly 21 columns (20 slots + dummy).
#include "fr_p1.cuh"

namespace fr {

bool p1_variant_k21(int ld, int threads, P1Variant* out) {
    return p1_k21_with(MkPlain{}, ld, threads, out);
}

}  // namespace fr
