// fr_p2_adj21.cu -- unrolled-gradient (adjoint) kernels for exactly 21 columns.
#include "fr_p2_adj.cuh"

namespace fr {

bool p2_adj_k21(int R, int threads, P2Variant* v) {
    switch (R) {
        case 8: p2::p2_make_adj<21, 8, true>(threads, v); return true;
        case 16: p2::p2_make_adj<21, 16, true>(threads, v); return true;
        case 24: p2::p2_make_adj<21, 24, true>(threads, v); return true;
        default: return false;
    }
}

}  // namespace fr
