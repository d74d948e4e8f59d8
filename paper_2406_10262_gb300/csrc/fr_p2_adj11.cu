// fr_p2_adj11.cu -- unrolled-gradient (adjoint) kernels for exactly 11 and 6 columns.
#include "fr_p2_adj.cuh"

namespace fr {

bool p2_adj_k11_k6(int nc, int R, int threads, P2Variant* v) {
    if (nc == 11) {
        switch (R) {
            case 8: p2::p2_make_adj<11, 8, true>(threads, v); return true;
            case 16: p2::p2_make_adj<11, 16, true>(threads, v); return true;
            case 24: p2::p2_make_adj<11, 24, true>(threads, v); return true;
            default: return false;
        }
    }
    if (nc == 6) {
        switch (R) {
            case 8: p2::p2_make_adj<6, 8, true>(threads, v); return true;
            case 16: p2::p2_make_adj<6, 16, true>(threads, v); return true;
            case 24: p2::p2_make_adj<6, 24, true>(threads, v); return true;
            default: return false;
        }
    }
    return false;
}

}  // namespace fr
