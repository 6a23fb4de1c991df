// D2Q9 time-step kernels, N = 5, 6, fp32 storage/arithmetic variant.
#include "nfe_fused2d.cuh"

namespace nfe {
const Ops *ops_d2q9_fp32_n56(int N) {
    if (N == 5) return ops_fused2d_one<5, float, float>(NFE_FP32); if (N == 6) return ops_fused2d_one<6, float, float>(NFE_FP32);
    return nullptr;
}
}  // namespace nfe
