// FP64 reductions of the fields written by k_moments (diagnostics, not on the
// time-step path).  Fixed block partition and order, so the result is
// deterministic for a given grid.
#include "nfe_kernels.cuh"

namespace nfe {

const char *kKernelNames[K_NKINDS] = {"fused_step", "moments", "reduce", "step_physics", "step_gather"};

// kind of diag value q: 0 = sum, 1 = sum of |.|, 2 = max |.|, 3 = min, 4 = max speed
__device__ __forceinline__ void diag_source(int q, int N, int &plane, int &kind) {
    if (q < N) { plane = q; kind = 0; return; }                        // mass
    if (q < N + 3) { plane = N + (q - N); kind = 0; return; }          // momentum
    if (q < N + 6) { plane = N + 4 + (q - N - 3); kind = 0; return; }  // sum F_s
    if (q < N + 9) { plane = N + 4 + (q - N - 6); kind = 1; return; }  // sum |F_s|
    if (q < 2 * N + 9) { plane = q - N - 9; kind = 2; return; }        // max |C|
    if (q < 3 * N + 9) { plane = q - 2 * N - 9; kind = 3; return; }    // min C
    plane = N; kind = 4;                                               // max speed
}

__device__ __forceinline__ double combine(int kind, double a, double b) {
    if (kind <= 1) return a + b;
    if (kind == 3) return fmin(a, b);
    return fmax(a, b);
}

__device__ __forceinline__ double identity(int kind) {
    if (kind <= 1) return 0.0;
    if (kind == 3) return 1.0e300;
    return 0.0;
}

__device__ double block_reduce(double v, int kind, double *sh) {
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) sh[t] = combine(kind, sh[t], sh[t + o]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void k_reduce_partial(long long n, int N, const double *__restrict__ fields,
                                 double *__restrict__ partials) {
    __shared__ double sh[256];
    const int nq = diag_count(N) - 1;   // the last value (nonfinite) comes from the flag
    for (int q = 0; q < nq; ++q) {
        int plane, kind;
        diag_source(q, N, plane, kind);
        double acc = identity(kind);
        for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
             s += (long long)gridDim.x * blockDim.x) {
            double val;
            if (kind == 4) {
                const double a = fields[size_t(N) * n + s], b = fields[size_t(N + 1) * n + s],
                             c = fields[size_t(N + 2) * n + s];
                val = sqrt(a * a + b * b + c * c);
            } else {
                val = fields[size_t(plane) * n + s];
                if (kind == 1 || kind == 2) val = fabs(val);
            }
            acc = combine(kind, acc, val);
        }
        const double r = block_reduce(acc, kind, sh);
        if (threadIdx.x == 0) partials[size_t(blockIdx.x) * nq + q] = r;
    }
}

__global__ void k_reduce_final(int nblocks, int N, const double *__restrict__ partials,
                               const int *__restrict__ flag, double *__restrict__ diag) {
    __shared__ double sh[256];
    const int nq = diag_count(N) - 1;
    for (int q = 0; q < nq; ++q) {
        int plane, kind;
        diag_source(q, N, plane, kind);
        double acc = identity(kind);
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) acc = combine(kind, acc, partials[size_t(b) * nq + q]);
        const double r = block_reduce(acc, kind, sh);
        if (threadIdx.x == 0) diag[q] = r;
    }
    if (threadIdx.x == 0) diag[nq] = double(*flag);
}

}  // namespace nfe
