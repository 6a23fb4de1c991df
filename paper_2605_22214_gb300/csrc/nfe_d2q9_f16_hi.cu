// D2Q9 time-step kernels, N = 5 .. 8, f16 storage/arithmetic variant.
#include "nfe_fused2d.cuh"

namespace nfe {
const Ops *ops_d2q9_f16_hi(int N) { return ops_fused2d_hi<float, __half>(N, NFE_FP32_F16STORE); }
}  // namespace nfe
