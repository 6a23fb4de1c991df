// D2Q9 time-step kernels, N = 2 .. 8, bf16 storage/arithmetic variant: the fused
// single-kernel step (three tile shapes) plus the shared helpers.
#include "nfe_fused2d.cuh"

namespace nfe {
const Ops *ops_d2q9_bf16(int N) { return ops_fused2d<float, __nv_bfloat16>(N, NFE_FP32_BF16STORE); }
}  // namespace nfe
