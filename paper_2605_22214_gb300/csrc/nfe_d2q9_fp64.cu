// D2Q9 time-step kernels, N = 2 .. 8, fp64 storage/arithmetic variant: the fused
// single-kernel step (three tile shapes) plus the shared helpers.
#include "nfe_fused2d.cuh"

namespace nfe {
const Ops *ops_d2q9_fp64(int N) { return ops_fused2d<double, double>(N, NFE_FP64); }
}  // namespace nfe
