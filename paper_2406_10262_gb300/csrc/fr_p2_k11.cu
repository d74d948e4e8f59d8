// fr_p2_k11.cu -- per-item parametrisation kernels compiled for exactly 11 columns.
#include "fr_p2.cuh"

namespace fr {

bool p2_variant_k11(int R, int threads, P2Variant* out) {
    switch (R) {
        case 8: *out = p2::p2_make<11, 8, true>(threads); return true;
        case 16: *out = p2::p2_make<11, 16, true>(threads); return true;
        case 24: *out = p2::p2_make<11, 24, true>(threads); return true;
        default: return false;
    }
}

}  // namespace fr
