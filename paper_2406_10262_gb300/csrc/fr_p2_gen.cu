// fr_p2_gen.cu -- per-item parametrisation kernels for padded column buckets (8 rows per thread).
#include "fr_p2.cuh"

namespace fr {

bool p2_variant_generic(int ncb, int threads, P2Variant* out) {
    switch (ncb) {
        case 8: *out = p2::p2_make<8, 8, false>(threads); return true;
        case 16: *out = p2::p2_make<16, 8, false>(threads); return true;
        case 32: *out = p2::p2_make<32, 8, false>(threads); return true;
        default: return false;
    }
}

}  // namespace fr
