// Allocation-free FP64 field statistics: a variant of the diagnostics
// reduction (k_reduce_partial / k_reduce_final) whose per-block partial
// results live in a file-scope device array instead of memory the library
// allocates.  For callers that cannot call cudaMalloc (for example code that
// runs inside another framework's memory pool or a pre-allocated arena, where
// an extra device allocation would fail or break the host's accounting).
//
// The array is global to the library: every GPU that loads libnfe holds it
// until the process exits, every call uses it, and it keeps the last call's
// contents.  Calls that overlap on the GPU (two streams, or a call still
// running when the next starts on another stream) race on it.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "nfe_internal.h"

namespace nfe {
namespace {

constexpr int kStatBlocks = 512;                 // blocks of the partial pass
constexpr int kStatMaxPlanes = NFE_STATS_MAX_PLANES;
constexpr int kStatPer = 4;                      // sum, sum |.|, max |.|, min

// 512 blocks x 16 planes x 4 values x 8 bytes = 256 KiB
__device__ __align__(256) double g_stat_scratch[kStatBlocks * kStatMaxPlanes * kStatPer];

// Largest / smallest value that lets a NaN through (fmax and fmin would drop it), so that a
// field holding a NaN reports NaN as its largest magnitude and its minimum.
__device__ __forceinline__ double nan_max(double a, double b) { return (a != a || b != b) ? NAN : fmax(a, b); }
__device__ __forceinline__ double nan_min(double a, double b) { return (a != a || b != b) ? NAN : fmin(a, b); }

__device__ __forceinline__ void stat_reduce(double (&v)[kStatPer], double *sh) {
    const int t = threadIdx.x;
    for (int j = 0; j < kStatPer; ++j) sh[j * blockDim.x + t] = v[j];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (t < o) {
            sh[0 * blockDim.x + t] += sh[0 * blockDim.x + t + o];
            sh[1 * blockDim.x + t] += sh[1 * blockDim.x + t + o];
            sh[2 * blockDim.x + t] = nan_max(sh[2 * blockDim.x + t], sh[2 * blockDim.x + t + o]);
            sh[3 * blockDim.x + t] = nan_min(sh[3 * blockDim.x + t], sh[3 * blockDim.x + t + o]);
        }
        __syncthreads();
    }
    for (int j = 0; j < kStatPer; ++j) v[j] = sh[j * blockDim.x];
    __syncthreads();
}

__global__ void k_stats_partial(int nplanes, long long n, const double *__restrict__ planes,
                                double *__restrict__ scratch) {
    __shared__ double sh[kStatPer * 256];
    for (int p = 0; p < nplanes; ++p) {
        double v[kStatPer] = {0.0, 0.0, 0.0, INFINITY};
        for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
             s += (long long)gridDim.x * blockDim.x) {
            const double x = planes[size_t(p) * n + s];
            v[0] += x;
            v[1] += fabs(x);
            v[2] = nan_max(v[2], fabs(x));
            v[3] = nan_min(v[3], x);
        }
        stat_reduce(v, sh);
        if (threadIdx.x == 0)
            for (int j = 0; j < kStatPer; ++j) scratch[(size_t(blockIdx.x) * kStatMaxPlanes + p) * kStatPer + j] = v[j];
    }
}

__global__ void k_stats_final(int nplanes, int nblocks, const double *__restrict__ scratch,
                              double *__restrict__ out) {
    __shared__ double sh[kStatPer * 256];
    for (int p = 0; p < nplanes; ++p) {
        double v[kStatPer] = {0.0, 0.0, 0.0, INFINITY};
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            const double *q = scratch + (size_t(b) * kStatMaxPlanes + p) * kStatPer;
            v[0] += q[0];
            v[1] += q[1];
            v[2] = nan_max(v[2], q[2]);
            v[3] = nan_min(v[3], q[3]);
        }
        stat_reduce(v, sh);
        if (threadIdx.x == 0)
            for (int j = 0; j < kStatPer; ++j) out[p * kStatPer + j] = v[j];
    }
}

// Device address of g_stat_scratch, looked up once per device with that device current.
std::mutex g_addr_mutex;
void *g_addr[64] = {nullptr};

}  // namespace
}  // namespace nfe

using namespace nfe;

extern "C" nfe_status nfe_field_stats_static(int nplanes, int64_t n, const double *d_planes, double *d_out,
                                             void *cuda_stream) {
    if (nplanes < 1 || nplanes > kStatMaxPlanes)
        return set_error(NFE_EINVAL, "nfe_field_stats_static: nplanes must be 1..16 (the static scratch holds 16 planes)");
    if (n < 1 || n > (int64_t(1) << 40)) return set_error(NFE_EINVAL, "nfe_field_stats_static: n must be 1..2^40");
    if (!d_planes || !d_out) return set_error(NFE_EINVAL, "nfe_field_stats_static: NULL pointer");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return set_error(NFE_ECUDA, "nfe_field_stats_static: no current CUDA device");
    }
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_addr_mutex);
        if (!g_addr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_stat_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return set_error(NFE_ECUDA, "nfe_field_stats_static: cudaGetSymbolAddress of the static scratch failed");
            }
            g_addr[dev] = ptr;
        }
        scratch = g_addr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const long long blocks_needed = (n + 255) / 256;
    const int nblocks = int(blocks_needed < kStatBlocks ? blocks_needed : kStatBlocks);
    k_stats_partial<<<nblocks, 256, 0, st>>>(nplanes, n, d_planes, static_cast<double *>(scratch));
    k_stats_final<<<1, 256, 0, st>>>(nplanes, nblocks, static_cast<const double *>(scratch), d_out);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(NFE_ECUDA, cudaGetErrorString(e));
    return NFE_OK;
}
