// D3Q19 time-step kernels, N = 5, 6, bf16 storage/arithmetic variant.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_bf16_n56(int N) {
    if (N == 5) return ops_fused3d_one<5, float, __nv_bfloat16>(NFE_FP32_BF16STORE); if (N == 6) return ops_fused3d_one<6, float, __nv_bfloat16>(NFE_FP32_BF16STORE);
    return nullptr;
}
}  // namespace nfe
