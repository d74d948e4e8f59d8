// fr_p1_k21.cu -- free-cost kernels compiled for exactly 21 columns (20 slots + dummy): the tile
// sweep with eight rows per thread, at a shared column stride of 512, 1024 or 2048 floats.
#include "fr_p1.cuh"

namespace fr {

bool p1_variant_k21(int ld, int threads, P1Variant* out) {
    if (ld <= 512)
        *out = make_variant<21, 8, true, 512>(threads);
    else if (ld <= 1024)
        *out = make_variant<21, 8, true, 1024>(threads);
    else if (ld <= 2048)
        *out = make_variant<21, 8, true, 2048>(threads);
    else
        return false;
    return true;
}

}  // namespace fr
