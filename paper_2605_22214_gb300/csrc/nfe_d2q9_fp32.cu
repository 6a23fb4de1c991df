// D2Q9 time-step kernels, N = 2 .. 8, fp32 storage/arithmetic variant.
#include "nfe_kernels.cuh"

namespace nfe {
const Ops *ops_d2q9_fp32(int N) { return ops_for_n<LD2Q9, float, float>(N, NFE_FP32); }
}  // namespace nfe
