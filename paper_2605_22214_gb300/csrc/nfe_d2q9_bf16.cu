// D2Q9 time-step kernels, N = 2 .. 8, bf16 storage/arithmetic variant.
#include "nfe_kernels.cuh"

namespace nfe {
const Ops *ops_d2q9_bf16(int N) { return ops_for_n<LD2Q9, float, __nv_bfloat16>(N, NFE_FP32_BF16STORE); }
}  // namespace nfe
