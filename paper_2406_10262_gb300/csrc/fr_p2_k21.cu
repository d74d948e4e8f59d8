// fr_p2_k21.cu -- per-item parametrisation kernels compiled for exactly 21 columns.
#include "fr_p2.cuh"

namespace fr {

bool p2_variant_k21(int R, int threads, P2Variant* out) {
    switch (R) {
        case 8: *out = p2::p2_make<21, 8, true>(threads); return true;
        case 16: *out = p2::p2_make<21, 16, true>(threads); return true;
        case 20: *out = p2::p2_make<21, 20, true>(threads); return true;
        case 24: *out = p2::p2_make<21, 24, true>(threads); return true;
        default: return false;
    }
}

}  // namespace fr
