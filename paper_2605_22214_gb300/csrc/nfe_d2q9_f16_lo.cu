// D2Q9 time-step kernels, N = 2 .. 4, f16 storage/arithmetic variant (the fused
// single-kernel step: three tile shapes, the stored-g and geometry forms), and the dispatch
// over N.
#include "nfe_fused2d.cuh"

namespace nfe {
const Ops *ops_d2q9_f16_n56(int N);
const Ops *ops_d2q9_f16_n78(int N);
const Ops *ops_d2q9_f16(int N) {
    if (N <= 4) return ops_fused2d_lo<float, __half>(N, NFE_FP32_F16STORE);
    return N <= 6 ? ops_d2q9_f16_n56(N) : ops_d2q9_f16_n78(N);
}
}  // namespace nfe
