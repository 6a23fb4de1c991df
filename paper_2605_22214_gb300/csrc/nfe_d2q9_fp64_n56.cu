// D2Q9 time-step kernels, N = 5, 6, fp64 storage/arithmetic variant.
#include "nfe_fused2d.cuh"

namespace nfe {
const Ops *ops_d2q9_fp64_n56(int N) {
    if (N == 5) return ops_fused2d_one<5, double, double>(NFE_FP64); if (N == 6) return ops_fused2d_one<6, double, double>(NFE_FP64);
    return nullptr;
}
}  // namespace nfe
