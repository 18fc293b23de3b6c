// Beam-search kernels over F32 traversal rows (instantiations of
// search_kernel.cuh, one translation unit per row type for parallel builds).
#include "search_kernel.cuh"

namespace esg_sk {

SearchFn pick_f32(int vpl, bool occ5) {
    if (occ5) return nullptr;   // FP32 rows spill at 96 registers
    switch (vpl) {
        case 1: return search_kernel<ESG_F32, 1>;
        case 2: return search_kernel<ESG_F32, 2>;
        case 3: return search_kernel<ESG_F32, 3>;
        case 4: return search_kernel<ESG_F32, 4>;
        case 6: return search_kernel<ESG_F32, 6>;
        case 8: return search_kernel<ESG_F32, 8>;
    }
    return nullptr;
}

}  // namespace esg_sk
