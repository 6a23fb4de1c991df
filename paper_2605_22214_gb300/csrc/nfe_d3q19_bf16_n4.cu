// D3Q19 time-step kernels, N = 4, bf16 storage/arithmetic variant.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_bf16_n4(int N) {
    if (N == 4) return ops_fused3d_one<4, float, __nv_bfloat16>(NFE_FP32_BF16STORE);
    return nullptr;
}
}  // namespace nfe
