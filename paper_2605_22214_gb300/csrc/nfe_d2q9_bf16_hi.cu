// D2Q9 time-step kernels, N = 5 .. 8, bf16 storage/arithmetic variant.
#include "nfe_fused2d.cuh"

namespace nfe {
const Ops *ops_d2q9_bf16_hi(int N) { return ops_fused2d_hi<float, __nv_bfloat16>(N, NFE_FP32_BF16STORE); }
}  // namespace nfe
