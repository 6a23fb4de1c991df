// D2Q9 time-step kernels, N = 2 .. 8, f16 storage/arithmetic variant.
#include "nfe_kernels.cuh"

namespace nfe {
const Ops *ops_d2q9_f16(int N) { return ops_for_n<LD2Q9, float, __half>(N, NFE_FP32_F16STORE); }
}  // namespace nfe
