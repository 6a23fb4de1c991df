// D3Q19 time-step kernels, N = 4, fp32 storage/arithmetic variant.
#include "nfe_fused3d.cuh"

namespace nfe {
const Ops *ops_d3q19_fp32_n4(int N) {
    if (N == 4) return ops_fused3d_one<4, float, float>(NFE_FP32);
    return nullptr;
}
}  // namespace nfe
