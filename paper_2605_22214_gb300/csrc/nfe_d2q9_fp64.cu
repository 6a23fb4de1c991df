// D2Q9 time-step kernels, N = 2 .. 8, fp64 storage/arithmetic variant.
#include "nfe_kernels.cuh"

namespace nfe {
const Ops *ops_d2q9_fp64(int N) { return ops_for_n<LD2Q9, double, double>(N, NFE_FP64); }
}  // namespace nfe
