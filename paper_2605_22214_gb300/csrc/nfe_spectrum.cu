// Domain size of the phase-separation study (Sec. IV, Eq. for L_i): for every
// component, lambda_i = H(C_i - 1/2), its discrete Fourier transform (cuFFT, a
// library step), and
//   L_i = 2 pi sum_{k != 0} |lambda_i(k)|^2 / sum_{k != 0} |k| |lambda_i(k)|^2,
// the integrals of S_i(k) = <lambda_i(k) lambda_i(-k)> over the k-plane written as
// sums over the modes of the grid (circular averaging does not change them).
// Optionally the circularly averaged S(k) of one component, in shells of width
// 2 pi / min(n_x, n_y[, n_z]).
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "nfe_spectrum.h"

namespace nfe {

namespace {

constexpr double kTwoPi = 6.283185307179586476925286766559;

__global__ void k_heaviside(long long n, const double *__restrict__ C, double *__restrict__ lam) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) lam[i] = C[i] >= 0.5 ? 1.0 : 0.0;
}

// One thread per stored mode of the real-to-complex transform (nx/2 + 1 per row).  Modes
// 0 < kx < nx/2 stand for themselves and their Hermitian partner (weight 2).  sums[0] +=
// sum w |F|^2, sums[1] += sum w |k| |F|^2 over k != 0; bins (2 nbins values, or null):
// per shell the weighted power and the mode count.
__global__ void k_spectrum_sums(int nx, int ny, int nz, const cufftDoubleComplex *__restrict__ F,
                                double *__restrict__ sums, int nbins, double dk, double *__restrict__ bins) {
    const int nxh = nx / 2 + 1;
    const long long total = (long long)nxh * ny * nz;
    double p0 = 0.0, p1 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int kx = int(i % nxh);
        const long long r = i / nxh;
        const int ky = int(r % ny), kz = int(r / ny);
        if (kx == 0 && ky == 0 && kz == 0) continue;
        const double w = (kx == 0 || (nx % 2 == 0 && kx == nx / 2)) ? 1.0 : 2.0;
        const int my = ky <= ny / 2 ? ky : ky - ny;
        const int mz = kz <= nz / 2 ? kz : kz - nz;
        const double ax = double(kx) / nx, ay = double(my) / ny, az = double(mz) / nz;
        const double kk = kTwoPi * sqrt(ax * ax + ay * ay + az * az);
        const double pw = F[i].x * F[i].x + F[i].y * F[i].y;
        p0 += w * pw;
        p1 += w * kk * pw;
        if (bins) {
            const int b = int(kk / dk + 0.5);
            if (b >= 1 && b <= nbins) {
                atomicAdd(&bins[2 * (b - 1)], w * pw);
                atomicAdd(&bins[2 * (b - 1) + 1], w);
            }
        }
    }
    __shared__ double s0[256], s1[256];
    s0[threadIdx.x] = p0;
    s1[threadIdx.x] = p1;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s0[threadIdx.x] += s0[threadIdx.x + o];
            s1[threadIdx.x] += s1[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicAdd(&sums[0], s0[0]);
        atomicAdd(&sums[1], s1[0]);
    }
}

}  // namespace

struct Spectrum {
    Geom g;
    cufftHandle plan = 0;
    bool has_plan = false;
    double *lam = nullptr;                 // lambda of one component (n)
    cufftDoubleComplex *F = nullptr;       // its transform ((nx/2 + 1) ny nz)
    double *sums = nullptr;                // 2 per component
    double *bins = nullptr;                // 2 per shell
    int bins_cap = 0;
};

nfe_status spectrum_create(const Geom &g, int N, Spectrum **out, std::string &err) {
    Spectrum *sp = new Spectrum();
    sp->g = g;
    const size_t n = size_t(g.n), nF = size_t(g.nx / 2 + 1) * g.ny * g.nz;
    cufftResult r = g.nz > 1 ? cufftPlan3d(&sp->plan, g.nz, g.ny, g.nx, CUFFT_D2Z)
                             : cufftPlan2d(&sp->plan, g.ny, g.nx, CUFFT_D2Z);
    if (r != CUFFT_SUCCESS) {
        delete sp;
        err = "cuFFT plan creation failed (code " + std::to_string(int(r)) + ")";
        return NFE_ECUDA;
    }
    sp->has_plan = true;
    cudaError_t e = cudaMalloc(&sp->lam, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&sp->F, nF * sizeof(cufftDoubleComplex));
    if (e == cudaSuccess) e = cudaMalloc(&sp->sums, 2 * size_t(N) * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        spectrum_destroy(sp);
        err = std::string("domain-size scratch: ") + cudaGetErrorString(e);
        return NFE_ENOMEM;
    }
    *out = sp;
    return NFE_OK;
}

void spectrum_destroy(Spectrum *sp) {
    if (!sp) return;
    if (sp->has_plan) cufftDestroy(sp->plan);
    cudaFree(sp->lam);
    cudaFree(sp->F);
    cudaFree(sp->sums);
    cudaFree(sp->bins);
    delete sp;
}

nfe_status domain_size(Spectrum *sp, int N, const double *C, int component, int nbins, double *L, double *Sk,
                       cudaStream_t st, std::string &err) {
    const Geom &g = sp->g;
    const long long n = g.n;
    if (nbins > sp->bins_cap) {
        cudaFree(sp->bins);
        sp->bins = nullptr;
        if (cudaMalloc(&sp->bins, 2 * size_t(nbins) * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            sp->bins_cap = 0;
            err = "domain-size bins: allocation failed";
            return NFE_ENOMEM;
        }
        sp->bins_cap = nbins;
    }
    if (cufftSetStream(sp->plan, st) != CUFFT_SUCCESS) { err = "cufftSetStream failed"; return NFE_ECUDA; }
    cudaError_t e = cudaMemsetAsync(sp->sums, 0, 2 * size_t(N) * sizeof(double), st);
    if (e == cudaSuccess && nbins > 0) e = cudaMemsetAsync(sp->bins, 0, 2 * size_t(nbins) * sizeof(double), st);
    if (e != cudaSuccess) { err = cudaGetErrorString(e); return NFE_ECUDA; }
    const int nmin = g.nz > 1 ? std::min(std::min(g.nx, g.ny), g.nz) : std::min(g.nx, g.ny);
    const double dk = kTwoPi / nmin;
    for (int c = 0; c < N; ++c) {
        k_heaviside<<<unsigned((n + 255) / 256), 256, 0, st>>>(n, C + size_t(c) * n, sp->lam);
        if (cufftExecD2Z(sp->plan, sp->lam, sp->F) != CUFFT_SUCCESS) { err = "cufftExecD2Z failed"; return NFE_ECUDA; }
        const bool want = c == component && nbins > 0;
        k_spectrum_sums<<<512, 256, 0, st>>>(g.nx, g.ny, g.nz, sp->F, sp->sums + 2 * c, want ? nbins : 0, dk,
                                             want ? sp->bins : nullptr);
    }
    std::vector<double> h(2 * size_t(N)), hb(2 * size_t(nbins));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), sp->sums, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && nbins > 0)
        e = cudaMemcpyAsync(hb.data(), sp->bins, hb.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { err = cudaGetErrorString(e); return NFE_ECUDA; }
    double sum = 0.0;
    int cnt = 0;
    for (int c = 0; c < N; ++c) {
        L[c] = h[2 * c + 1] > 0.0 ? kTwoPi * h[2 * c] / h[2 * c + 1] : NAN;   // no interface: undefined
        if (std::isfinite(L[c])) { sum += L[c]; ++cnt; }
    }
    L[N] = cnt > 0 ? sum / cnt : NAN;
    for (int b = 0; b < nbins; ++b) Sk[b] = hb[2 * b + 1] > 0.0 ? hb[2 * b] / hb[2 * b + 1] : 0.0;
    return NFE_OK;
}

}  // namespace nfe
