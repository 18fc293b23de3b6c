// Beam-search kernels over FP8 traversal rows (instantiations of
// search_kernel.cuh, one translation unit per row type for parallel builds).
#include "search_kernel.cuh"

namespace esg_sk {

SearchFn pick_fp8(int vpl, bool occ5) {
    if (occ5) {   // at most 96 registers without spills for these splits
        if (vpl == 1) return search_kernel<ESG_FP8E4M3, 1, 5>;
        if (vpl == 3) return search_kernel<ESG_FP8E4M3, 3, 5>;
        return nullptr;
    }
    switch (vpl) {
        case 1: return search_kernel<ESG_FP8E4M3, 1>;
        case 2: return search_kernel<ESG_FP8E4M3, 2>;
        case 3: return search_kernel<ESG_FP8E4M3, 3>;
    }
    return nullptr;
}

}  // namespace esg_sk
