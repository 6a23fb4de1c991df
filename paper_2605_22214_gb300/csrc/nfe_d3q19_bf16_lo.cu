// D3Q19 time-step kernels, N = 2, 3, bf16 storage/arithmetic variant, and the dispatch over N
// (N = 4, 5..6 and 7..8 are compiled in their own translation units, in parallel).
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_bf16_n4(int N);
const Ops *ops_d3q19_bf16_n56(int N);
const Ops *ops_d3q19_bf16_n78(int N);
const Ops *ops_d3q19_bf16(int N) {
    switch (N) {
        case 2: return ops_fused3d_one<2, float, __nv_bfloat16>(NFE_FP32_BF16STORE);
        case 3: return ops_fused3d_one<3, float, __nv_bfloat16>(NFE_FP32_BF16STORE);
        case 4: return ops_d3q19_bf16_n4(N);
        case 5: case 6: return ops_d3q19_bf16_n56(N);
        case 7: case 8: return ops_d3q19_bf16_n78(N);
        default: return nullptr;
    }
}
}  // namespace nfe
