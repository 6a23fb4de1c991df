// D3Q19 time-step kernels, N = 4, f16 storage/arithmetic variant.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_f16_n4(int N) {
    if (N == 4) return ops_fused3d_one<4, float, __half>(NFE_FP32_F16STORE);
    return nullptr;
}
}  // namespace nfe
