// D3Q19 time-step kernels, N = 7, 8, bf16 storage/arithmetic variant.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_bf16_n78(int N) {
    if (N == 7) return ops_fused3d_one<7, float, __nv_bfloat16>(NFE_FP32_BF16STORE); if (N == 8) return ops_fused3d_one<8, float, __nv_bfloat16>(NFE_FP32_BF16STORE);
    return nullptr;
}
}  // namespace nfe
