// D2Q9 time-step kernels, N = 5 .. 8, fp64 storage/arithmetic variant.
#include "nfe_fused2d.cuh"

namespace nfe {
const Ops *ops_d2q9_fp64_hi(int N) { return ops_fused2d_hi<double, double>(N, NFE_FP64); }
}  // namespace nfe
