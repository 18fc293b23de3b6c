// Beam-search kernels over BF16 traversal rows (instantiations of
// search_kernel.cuh, one translation unit per row type for parallel builds).
#include "search_kernel.cuh"

namespace esg_sk {

SearchFn pick_bf16(int vpl, bool occ5) {
    if (occ5) {   // 96 registers without spills for these splits
        if (vpl == 3) return search_kernel<ESG_BF16, 3, 5>;
        if (vpl == 6) return search_kernel<ESG_BF16, 6, 5>;
        return nullptr;
    }
    switch (vpl) {
        case 1: return search_kernel<ESG_BF16, 1>;
        case 2: return search_kernel<ESG_BF16, 2>;
        case 3: return search_kernel<ESG_BF16, 3>;
        case 4: return search_kernel<ESG_BF16, 4>;
        case 6: return search_kernel<ESG_BF16, 6>;
    }
    return nullptr;
}

}  // namespace esg_sk
