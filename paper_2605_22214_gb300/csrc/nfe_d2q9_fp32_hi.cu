// D2Q9 time-step kernels, N = 5 .. 8, fp32 storage/arithmetic variant.
#include "nfe_fused2d.cuh"

namespace nfe {
const Ops *ops_d2q9_fp32_hi(int N) { return ops_fused2d_hi<float, float>(N, NFE_FP32); }
}  // namespace nfe
