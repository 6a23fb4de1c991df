// Shared device code of the N-component free-energy LBM (arXiv 2605.22214):
// lattices (D2Q9, D3Q19), storage formats of f, the bulk energy E_B (Eq. 5), the
// factored flux potential S_i = C_i q_i(C) + (3D/4) lap C_i (Eq. 12), a generic
// site stencil, the viscosity rule (Eq. 42), and the non-step kernels: fields of
// the current state (moments), initialisation, (un)packing and FP64 reductions.
// The time-step kernels are in nfe_fused2d.cuh (D2Q9) and nfe_fused3d.cuh (D3Q19).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

#include "nfe_internal.h"

namespace nfe {

// ----------------------------------------------------------------------------
// Lattices.  D2Q9 in the order of Eqs. 20-21; D3Q19 in the standard set
// (axis pairs, then the xy, xz and yz diagonals).  In both, the opposite of
// an odd k is k + 1.
// ----------------------------------------------------------------------------
struct LD2Q9 {
    static constexpr int Q = 9, D = 2;
    __host__ __device__ static constexpr int ex(int k) {
        return k == 1 || k == 5 || k == 7 ? 1 : (k == 2 || k == 6 || k == 8 ? -1 : 0);
    }
    __host__ __device__ static constexpr int ey(int k) {
        return k == 3 || k == 5 || k == 8 ? 1 : (k == 4 || k == 6 || k == 7 ? -1 : 0);
    }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr double w(int k) { return k == 0 ? 4.0 / 9.0 : (k < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }
};

struct LD3Q19 {
    static constexpr int Q = 19, D = 3;
    // velocity k as (ex, ey, ez)
    __host__ __device__ static constexpr int ex(int k) {
        return (k == 1 || k == 7 || k == 9 || k == 11 || k == 13) ? 1
             : (k == 2 || k == 8 || k == 10 || k == 12 || k == 14) ? -1 : 0;
    }
    __host__ __device__ static constexpr int ey(int k) {
        return (k == 3 || k == 7 || k == 10 || k == 15 || k == 17) ? 1
             : (k == 4 || k == 8 || k == 9 || k == 16 || k == 18) ? -1 : 0;
    }
    __host__ __device__ static constexpr int ez(int k) {
        return (k == 5 || k == 11 || k == 14 || k == 15 || k == 18) ? 1
             : (k == 6 || k == 12 || k == 13 || k == 16 || k == 17) ? -1 : 0;
    }
    __host__ __device__ static constexpr double w(int k) { return k == 0 ? 1.0 / 3.0 : (k < 7 ? 1.0 / 18.0 : 1.0 / 36.0); }
};

__host__ __device__ constexpr int opp(int k) { return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1); }

// Compile-time loop: calls f(std::integral_constant<int, i>) for i = B, B + S, ... < E, so that
// the lattice direction is a constant expression in the body.
template <int B, int E, int S, typename F>
__device__ __forceinline__ void sfor(F &&f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        sfor<B + S, E, S>(f);
    }
}

// ----------------------------------------------------------------------------
// Storage of f.  FP16 keeps f_k / w_k * 2^scale_exp, BF16 keeps f_k / w_k:
// in the pressure-based scheme f_k ~ w_k (3P + 3 e.v + ...) is already a
// deviation from rest, so dividing by w_k brings every direction to one scale.
// ----------------------------------------------------------------------------
template <typename S, typename T> struct FStore;
template <typename T> struct FStore<double, T> {
    __device__ static T load(const double *p, double, T) { return T(*p); }
    __device__ static void store(double *p, T v, double, T) { *p = double(v); }
};
template <typename T> struct FStore<float, T> {
    __device__ static T load(const float *p, double, T) { return T(*p); }
    __device__ static void store(float *p, T v, double, T) { *p = float(v); }
};
template <> struct FStore<__half, float> {
    __device__ static float load(const __half *p, double w, float finv) { return __half2float(*p) * (float(w) * finv); }
    __device__ static void store(__half *p, float v, double w, float fscale) { *p = __float2half_rn(v * (float(1.0 / w) * fscale)); }
};
template <> struct FStore<__nv_bfloat16, float> {
    __device__ static float load(const __nv_bfloat16 *p, double w, float) { return __bfloat162float(*p) * float(w); }
    __device__ static void store(__nv_bfloat16 *p, float v, double w, float) { *p = __float2bfloat16_rn(v * float(1.0 / w)); }
};

// ----------------------------------------------------------------------------
// Site helpers
// ----------------------------------------------------------------------------

// Index of x + e_k, or -1 when x + e_k lies beyond a wall.
template <class L>
__device__ __forceinline__ int neighbour(const Geom &g, int x, int y, int z, int k) {
    int xx = x + L::ex(k), yy = y + L::ey(k), zz = z + L::ez(k);
    if (L::ex(k) != 0) {
        if (xx < 0) { if (g.wx) return -1; xx += g.nx; }
        else if (xx >= g.nx) { if (g.wx) return -1; xx -= g.nx; }
    }
    if (L::ey(k) != 0) {
        if (yy < 0) { if (g.wy) return -1; yy += g.ny; }
        else if (yy >= g.ny) { if (g.wy) return -1; yy -= g.ny; }
    }
    if (L::ez(k) != 0) {
        if (zz < 0) { if (g.wz) return -1; zz += g.nz; }
        else if (zz >= g.nz) { if (g.wz) return -1; zz -= g.nz; }
    }
    return xx + g.nx * (yy + g.ny * zz);
}

template <int N, typename T>
__device__ __forceinline__ T bulk_energy(const T (&c)[N], const Coef<T> &cf) {
    // E_B = sum_{a<b} beta_ab [f(C_a) + f(C_b) - f(C_a + C_b)], f(C) = C^2 (1 - C)^2 (Eq. 5)
    T fw[N];
#pragma unroll
    for (int a = 0; a < N; ++a) { T u = c[a] * (T(1) - c[a]); fw[a] = u * u; }
    T E = T(0);
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = a + 1; b < N; ++b) {
            T t = c[a] + c[b];
            T u = t * (T(1) - t);
            E += cf.beta[a][b] * (fw[a] + fw[b] - u * u);
        }
    return E;
}

// Where the coefficients of the quartic (stabiliser) part of q are read (the part is skipped
// when cf.has_q4 is 0): device memory, or the kernel's parameter block when N <= kQ4InlineMaxN
// (saves a load per term; the D3Q19 step gains, while in the D2Q9 step the extra register
// pressure costs more than it saves).  Q4_ABSENT compiles no quartic code at all, for kernels
// launched only when Omega = 0: even never-executed quartic code raises register pressure.
// Q4_NOPHI reads the quartic part from device memory and adds the no-phi remainder (below).
enum Q4Source { Q4_GLOBAL = 0, Q4_PARAM = 1, Q4_ABSENT = 2, Q4_NOPHI = 3 };

template <int N, typename T, int Q4 = Q4_GLOBAL>
__device__ __forceinline__ void flux_poly(const T (&c)[N], const Coef<T> &cf, T (&q)[N - 1]) {
    // q_e(C): degree-2 monomials C_a C_b (a <= b) in nested-loop order, and the
    // structured quartic stabiliser part when Omega != 0.
#pragma unroll
    for (int e = 0; e < N - 1; ++e) q[e] = T(0);
    int idx = 0;
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
        for (int b = a; b < N; ++b) {
            T p = c[a] * c[b];
#pragma unroll
            for (int e = 0; e < N - 1; ++e) q[e] += cf.q2[e][idx] * p;
            ++idx;
        }
    if (Q4 != Q4_ABSENT && cf.has_q4) {
        // structured quartic part (layout in nfe_internal.h): a_{ilm} then b_{ikl} per i
        constexpr int M4 = mono4s_count(N);
        const auto coef = [&](int t) -> T {
            if constexpr (Q4 == Q4_PARAM && N <= kQ4InlineMaxN) return cf.q4c[t];
            else return __ldg(cf.q4 + t);
        };
        T sq[N];
#pragma unroll
        for (int a = 0; a < N; ++a) sq[a] = c[a] * c[a];
#pragma unroll
        for (int e = 0; e < N - 1; ++e) {
            int j = e * M4;
            T sa = T(0), sb = T(0);
#pragma unroll
            for (int l = 0; l < N; ++l) {
                if (l == e) continue;
                T lin = T(0);
#pragma unroll
                for (int m = 0; m < N; ++m) if (m != e && m != l) lin += coef(j++) * c[m];
                sa += sq[l] * lin;
            }
#pragma unroll
            for (int k = 0; k < N; ++k)
#pragma unroll
                for (int l = k + 1; l < N; ++l)
                    if (k != e && l != e) sb += coef(j++) * (sq[k] * sq[l]);
            q[e] += c[e] * sa + sb;
        }
    }
}

// The no-phi ablation: S_e += r_e(C), the cubic part of sum_j alpha_ej dE_B/dC_j (Eq. 12 without
// phi_j) that has no factor C_e, monomials a <= b <= d over the components other than e.
template <int N, typename T, int Q4>
__device__ __forceinline__ void flux_rest(const T (&c)[N], const Coef<T> &cf, T (&S)[N - 1]) {
    if constexpr (Q4 == Q4_NOPHI) {
        constexpr int M3 = mono3r_count(N);
#pragma unroll
        for (int e = 0; e < N - 1; ++e) {
            int j = e * M3;
            T r = T(0);
#pragma unroll
            for (int a = 0; a < N; ++a)
#pragma unroll
                for (int b = a; b < N; ++b)
#pragma unroll
                    for (int d = b; d < N; ++d)
                        if (a != e && b != e && d != e) r += __ldg(cf.r3 + j++) * (c[a] * c[b] * c[d]);
            S[e] += r;
        }
    }
}

// Stencil pass at one site: all N volume fractions at x, their grad and
// Laplacian (Eqs. 35-36) with the wall rule (a neighbour inside a wall takes
// the value at x, Sec. III C), grad E_B, and the neighbour indices.
template <class L, int N, typename T>
struct Stencil {
    T c[N];
    T lap[N];
    T gr[N][3];
    T gE[3];
    int nb[L::Q];
};

template <class L, int N, typename T>
__device__ __forceinline__ void stencil(const Geom &g, const Coef<T> &cf, const T *__restrict__ C,
                                        int s, int x, int y, int z, Stencil<L, N, T> &st,
                                        const unsigned char *__restrict__ node = nullptr,
                                        const T *__restrict__ ghost = nullptr) {
    const size_t n = size_t(g.n);
    T rest = T(0);
#pragma unroll
    for (int a = 0; a < N - 1; ++a) { st.c[a] = C[a * n + s]; rest += st.c[a]; }
    st.c[N - 1] = T(1) - rest;
    const T E0 = bulk_energy<N, T>(st.c, cf);
#pragma unroll
    for (int a = 0; a < N; ++a) { st.lap[a] = T(0); st.gr[a][0] = st.gr[a][1] = st.gr[a][2] = T(0); }
    st.gE[0] = st.gE[1] = st.gE[2] = T(0);
    st.nb[0] = s;
#pragma unroll
    for (int k = 1; k < L::Q; ++k) {
        const int j = neighbour<L>(g, x, y, z, k);
        st.nb[k] = j;
        if (j < 0) continue;               // wall: psi(x + e_k) := psi(x), difference 0
        // with an outflow, column nx - 1 sees the ghost column beyond it (solid where column
        // nx - 1 of that line is)
        const bool gcol = ghost && x == g.nx - 1 && L::ex(k) > 0;
        const int jrow = j / g.nx;
        if (node && node[gcol ? (g.nx - 1) + g.nx * jrow : j] == kNodeSolid) continue;   // solid node: the same rule
        T cn[N];
        T r2 = T(0);
#pragma unroll
        for (int a = 0; a < N - 1; ++a) {
            cn[a] = gcol ? ghost[size_t(a) * (g.ny * g.nz) + jrow] : C[a * n + j];
            r2 += cn[a];
        }
        cn[N - 1] = T(1) - r2;
        const T wk = T(L::w(k));
#pragma unroll
        for (int a = 0; a < N; ++a) {
            const T d = cn[a] - st.c[a];
            st.lap[a] += wk * d;
            if (L::ex(k)) st.gr[a][0] += (L::ex(k) > 0 ? wk : -wk) * d;
            if (L::ey(k)) st.gr[a][1] += (L::ey(k) > 0 ? wk : -wk) * d;
            if (L::ez(k)) st.gr[a][2] += (L::ez(k) > 0 ? wk : -wk) * d;
        }
        const T dE = bulk_energy<N, T>(cn, cf) - E0;
        if (L::ex(k)) st.gE[0] += (L::ex(k) > 0 ? wk : -wk) * dE;
        if (L::ey(k)) st.gE[1] += (L::ey(k) > 0 ? wk : -wk) * dE;
        if (L::ez(k)) st.gE[2] += (L::ez(k) > 0 ? wk : -wk) * dE;
    }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        st.lap[a] *= T(6);                 // 2 / c_s^2
        st.gr[a][0] *= T(3); st.gr[a][1] *= T(3); st.gr[a][2] *= T(3);   // 1 / c_s^2
    }
    st.gE[0] *= T(3); st.gE[1] *= T(3); st.gE[2] *= T(3);
}

// F_s (Eq. 34, or Eq. 31 when cf.nonconservative) and the flux potential S.
template <class L, int N, typename T>
__device__ __forceinline__ void force_and_potential(const Coef<T> &cf, const Stencil<L, N, T> &st,
                                                    T (&Fs)[3], T (&S)[N - 1]) {
    if (!cf.nonconservative) {
        Fs[0] = st.gE[0]; Fs[1] = st.gE[1]; Fs[2] = st.gE[2];
#pragma unroll
        for (int a = 0; a < N; ++a) {
            T h = T(0);
#pragma unroll
            for (int b = 0; b < N; ++b) if (b != a) h += cf.kappa[a][b] * st.lap[b];
            Fs[0] += h * st.gr[a][0]; Fs[1] += h * st.gr[a][1]; Fs[2] += h * st.gr[a][2];
        }
    } else {
        // mu_a = sum_{b != a} beta_ab (f'(C_a) - f'(C_a + C_b)) + kappa_ab lap C_b (Eq. 7)
        Fs[0] = Fs[1] = Fs[2] = T(0);
#pragma unroll
        for (int a = 0; a < N; ++a) {
            const T ca = st.c[a];
            const T fpa = T(2) * ca * (T(1) - T(3) * ca + T(2) * ca * ca);
            T mu = T(0);
#pragma unroll
            for (int b = 0; b < N; ++b) if (b != a) {
                const T t = ca + st.c[b];
                const T fpt = T(2) * t * (T(1) - T(3) * t + T(2) * t * t);
                mu += cf.beta[a][b] * (fpa - fpt) + cf.kappa[a][b] * st.lap[b];
            }
            Fs[0] += mu * st.gr[a][0]; Fs[1] += mu * st.gr[a][1]; Fs[2] += mu * st.gr[a][2];
        }
    }
    T q[N - 1];
    flux_poly<N, T>(st.c, cf, q);
#pragma unroll
    for (int e = 0; e < N - 1; ++e) S[e] = st.c[e] * q[e] + cf.d34 * st.lap[e];
}

// omega+ / omega- of the component with the largest C (Eq. 42); ties go to the
// lowest user index.
template <int N, typename T>
__device__ __forceinline__ void relaxation(const Coef<T> &cf, const T (&c)[N], T &op, T &om) {
    op = cf.omp[0]; om = cf.omm[0];
    if (cf.uniform_tau) return;           // one relaxation time for every component: nothing to choose
    T best = c[0];
    int bu = cf.uidx[0];
#pragma unroll
    for (int a = 1; a < N; ++a) {
        if (c[a] > best || (c[a] == best && cf.uidx[a] < bu)) {
            best = c[a]; bu = cf.uidx[a]; op = cf.omp[a]; om = cf.omm[a];
        }
    }
}

// ----------------------------------------------------------------------------
// Kernels
// ----------------------------------------------------------------------------

// Fields of the current state in FP64: C (N planes, user order), v (3), P, F_s (3).  With node
// classes (fluid and solid nodes only): the solid rule in the stencil, v = P = F_s = 0 on solid
// nodes.
template <class L, int N, typename T, typename SF>
__global__ void __launch_bounds__(256)
k_moments(Geom g, Coef<T> cf, const SF *__restrict__ fin, const T *__restrict__ C,
          double *__restrict__ out, int *__restrict__ flag, const unsigned char *__restrict__ node,
          const T *__restrict__ inl, const T *__restrict__ ghost) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    const int x = s % g.nx;
    const int r = s / g.nx;
    const int y = r % g.ny;
    const int z = r / g.ny;
    const size_t n = size_t(g.n);
    Stencil<L, N, T> st;
    stencil<L, N, T>(g, cf, C, s, x, y, z, st, node, ghost);
    T Fs[3], S[N - 1];
    force_and_potential<L, N, T>(cf, st, Fs, S);
    T sumf = T(0), j0 = T(0), j1 = T(0), j2 = T(0);
    bool bad = false;
#pragma unroll
    for (int k = 1; k < L::Q; ++k) {
        const T fk = FStore<SF, T>::load(fin + (k - 1) * n + s, L::w(k), cf.finv);
        bad |= !isfinite(fk);
        sumf += fk;
        if (L::ex(k)) j0 += L::ex(k) > 0 ? fk : -fk;
        if (L::ey(k)) j1 += L::ey(k) > 0 ? fk : -fk;
        if (L::ez(k)) j2 += L::ez(k) > 0 ? fk : -fk;
    }
    T cc = T(0);                          // body force on one component, F += C_c F_c
#pragma unroll
    for (int a = 0; a < N; ++a) cc += cf.fcsel[a] * st.c[a];
    T v0 = j0 + T(0.5) * (Fs[0] + cf.fb[0] + cc * cf.fc[0]);
    T v1 = j1 + T(0.5) * (Fs[1] + cf.fb[1] + cc * cf.fc[1]);
    T v2 = j2 + T(0.5) * (Fs[2] + cf.fb[2] + cc * cf.fc[2]);
    const T w0 = T(L::w(0));
    T P = (sumf - T(1.5) * w0 * (v0 * v0 + v1 * v1 + v2 * v2)) * T(1.0 / (3.0 * (1.0 - L::w(0))));
    if (node && node[s] != kNodeFluid) {
        v0 = v1 = v2 = P = Fs[0] = Fs[1] = Fs[2] = T(0);
        if (node[s] >= kNodeInlet0) {       // D3Q19 inlet row: v_b first
            const T *row = inl + (node[s] - kNodeInlet0) * (2 * N + 1);
            v0 = row[0]; v1 = row[1]; v2 = row[2];
        }
    }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        out[size_t(cf.uidx[a]) * n + s] = double(st.c[a]);
        bad |= !isfinite(st.c[a]);
    }
    out[(N + 0) * n + s] = double(v0);
    out[(N + 1) * n + s] = double(v1);
    out[(N + 2) * n + s] = double(v2);
    out[(N + 3) * n + s] = double(P);
    out[(N + 4) * n + s] = double(Fs[0]);
    out[(N + 5) * n + s] = double(Fs[1]);
    out[(N + 6) * n + s] = double(Fs[2]);
    if (bad) atomicOr(flag, 1);
}

// Link mask of every site of a D3Q19 geometry (solid and inlet nodes, convective outflow): bit k
// (k = 1..18) when x + e_k is a solid node (periodic wrap; a neighbour beyond an edge wall sets no
// bit, the wall mask covers it), bits 19..25 the class of x when x is not a fluid node, bit 29
// when x lies in the outflow column nx - 1 (its links with e_kx > 0 end in the ghost column, solid
// where column nx - 1 is), bit 30 when a neighbour is an inlet node, bit 31 when x is not a fluid
// node.
constexpr unsigned kLinkSolidBits = 0x7FFFEu, kLinkOutflowCol = 1u << 29, kLinkInletNear = 1u << 30,
                   kLinkNonFluid = 1u << 31;
__device__ __forceinline__ unsigned link_class(unsigned m) { return (m >> 19) & 0x7Fu; }

template <class L>
__global__ void k_link_mask(Geom g, const unsigned char *__restrict__ node, unsigned *__restrict__ out, int outflow) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    const int x = s % g.nx;
    const int r = s / g.nx;
    const int y = r % g.ny;
    const int z = r / g.ny;
    const unsigned cls = node[s];
    unsigned m = cls != kNodeFluid ? (kLinkNonFluid | (cls << 19)) : 0u;
    const bool ocol = outflow && x == g.nx - 1;
    if (ocol) m |= kLinkOutflowCol;
#pragma unroll
    for (int k = 1; k < L::Q; ++k) {
        const int j = neighbour<L>(g, x, y, z, k);
        if (j < 0) continue;
        if (ocol && L::ex(k) > 0) {
            // the ghost column: solid where column nx - 1 of that line is
            if (node[(g.nx - 1) + g.nx * (j / g.nx)] == kNodeSolid) m |= 1u << k;
            continue;
        }
        if (node[j] == kNodeSolid) m |= 1u << k;
        else if (node[j] >= kNodeInlet0) m |= kLinkInletNear;
    }
    out[s] = m;
}

// Ghost column of the convective outflow from column nx - 1 of buffer cur (rows = ny nz lines).
template <int N, typename T>
__global__ void k_ghost_init(Geom g, const T *__restrict__ C, T *__restrict__ ghost) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int rows = g.ny * g.nz;
    if (r >= rows) return;
#pragma unroll
    for (int e = 0; e < N - 1; ++e) ghost[size_t(e) * rows + r] = C[size_t(e) * size_t(g.n) + size_t(g.nx - 1) + size_t(g.nx) * r];
}

// D3Q19 inlet table: rows K x (3 + N) FP64 (v_b, C_b in internal order); out: K x (2N + 1) in the
// compute type: v_b (3), C_b of the evolved components, S_b (Eq. 12 at the uniform C_b).
template <int N, typename T>
__global__ void k_inlet_table3(Coef<T> cf, const double *__restrict__ rows, int K, T *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= K) return;
    const double *r = rows + size_t(j) * (3 + N);
    T c[N];
#pragma unroll
    for (int a = 0; a < N; ++a) c[a] = T(r[3 + a]);
    T q[N - 1], S[N - 1];
    flux_poly<N, T, Q4_GLOBAL>(c, cf, q);
#pragma unroll
    for (int e = 0; e < N - 1; ++e) S[e] = c[e] * q[e];
    flux_rest<N, T, Q4_GLOBAL>(c, cf, S);
    T *o = out + size_t(j) * (2 * N + 1);
    o[0] = T(r[0]); o[1] = T(r[1]); o[2] = T(r[2]);
#pragma unroll
    for (int e = 0; e < N - 1; ++e) { o[3 + e] = c[e]; o[N + 2 + e] = S[e]; }
}

// C := C_b on the inlet nodes of a D3Q19 geometry.
template <int N, typename T>
__global__ void k_inlet_fill3(Geom g, const unsigned char *__restrict__ node, const T *__restrict__ inl,
                              T *__restrict__ C) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    const unsigned char cls = node[s];
    if (cls < kNodeInlet0) return;
    const T *row = inl + (cls - kNodeInlet0) * (2 * N + 1);
#pragma unroll
    for (int e = 0; e < N - 1; ++e) C[size_t(e) * size_t(g.n) + s] = row[3 + e];
}

// f = f^eq(P = 0, v): f_k = s_k(v) for k >= 1 (Eqs. 27-28).
template <class L, typename T, typename SF>
__global__ void k_init_f(Geom g, Coef<T> cf, const double *__restrict__ v, SF *__restrict__ f) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    const size_t n = size_t(g.n);
    const double a0 = v[s], a1 = v[n + s], a2 = v[2 * n + s];
    const double uu = a0 * a0 + a1 * a1 + a2 * a2;
#pragma unroll
    for (int k = 1; k < L::Q; ++k) {
        const double eu = L::ex(k) * a0 + L::ey(k) * a1 + L::ez(k) * a2;
        const double sk = L::w(k) * (3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
        FStore<SF, T>::store(f + (k - 1) * n + s, T(sk), L::w(k), cf.fscale);
    }
}

// Stored-g path (tau_g != 1): g = g^eq(C, v, S(C)) at the start (Eq. 40 as read: the C_i part
// of the zeroth moment in the rest population, g^eq_k = C_i (delta_k0 + s_k(v)) + (1 - w_0) m S_i
// for k = 0 and - w_k m S_i otherwise), from the C of the state and an FP64 velocity (null: 0).
// Layout of g: plane (e Q + k) for evolved slot e and direction k.
template <class L, int N, typename T>
__global__ void k_init_g(Geom g, Coef<T> cf, const T *__restrict__ C, const double *__restrict__ v,
                         T *__restrict__ gout) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    const int x = s % g.nx;
    const int r = s / g.nx;
    const int y = r % g.ny;
    const int z = r / g.ny;
    const size_t n = size_t(g.n);
    Stencil<L, N, T> st;
    stencil<L, N, T>(g, cf, C, s, x, y, z, st);
    T Fs[3], S[N - 1];
    force_and_potential<L, N, T>(cf, st, Fs, S);
    const T a0 = v ? T(v[s]) : T(0), a1 = v ? T(v[n + s]) : T(0), a2 = v ? T(v[2 * n + s]) : T(0);
    const T uu = a0 * a0 + a1 * a1 + a2 * a2;
#pragma unroll
    for (int k = 0; k < L::Q; ++k) {
        const T wk = T(L::w(k));
        const T eu = T(L::ex(k)) * a0 + T(L::ey(k)) * a1 + T(L::ez(k)) * a2;
        const T sk = wk * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * uu);
#pragma unroll
        for (int e = 0; e < N - 1; ++e) {
            const T geq = k == 0 ? st.c[e] * (T(1) + sk) + (T(1) - wk) * cf.m * S[e] : st.c[e] * sk - wk * cf.m * S[e];
            gout[(size_t(e) * L::Q + k) * n + s] = geq;
        }
    }
}

template <class L, typename T, typename SF>
__global__ void k_unpack_f(Geom g, Coef<T> cf, const SF *__restrict__ f, double *__restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    const size_t n = size_t(g.n);
#pragma unroll
    for (int k = 1; k < L::Q; ++k)
        out[(k - 1) * n + s] = double(FStore<SF, T>::load(f + (k - 1) * n + s, L::w(k), cf.finv));
}

template <typename T>
__global__ void k_pack_C(long long total, const double *__restrict__ in, T *__restrict__ out) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < total) out[i] = T(in[i]);
}

// FP64 reductions.  Block partials of diag_count(N) values, then one block
// combines them.  Layout as in nfe_internal.h.
__global__ void k_reduce_partial(long long n, int N, const double *__restrict__ fields,
                                 double *__restrict__ partials);
__global__ void k_reduce_final(int nblocks, int N, const double *__restrict__ partials,
                               const int *__restrict__ flag, double *__restrict__ diag);

// ----------------------------------------------------------------------------
// Launchers
// ----------------------------------------------------------------------------

inline unsigned blocks_for(long long n, int bs) { return unsigned((n + bs - 1) / bs); }

// Launchers of the non-step kernels for one lattice, N and precision.
template <class L, int N, typename T, typename SF>
struct Launch {
    static cudaError_t moments(const Geom &g, const void *coef, const Buffers &b, int cur, cudaStream_t st) {
        const Coef<T> &cf = *static_cast<const Coef<T> *>(coef);
        k_moments<L, N, T, SF><<<blocks_for(g.n, 256), 256, 0, st>>>(
            g, cf, static_cast<const SF *>(b.f[cur]), static_cast<const T *>(b.C[cur]), b.fields, b.flag, nullptr,
            nullptr, nullptr);
        return cudaGetLastError();
    }
    // with the node classes of a D3Q19 geometry (solid and inlet nodes)
    static cudaError_t moments_solid(const Geom &g, const void *coef, const Buffers &b, int cur, cudaStream_t st) {
        const Coef<T> &cf = *static_cast<const Coef<T> *>(coef);
        k_moments<L, N, T, SF><<<blocks_for(g.n, 256), 256, 0, st>>>(
            g, cf, static_cast<const SF *>(b.f[cur]), static_cast<const T *>(b.C[cur]), b.fields, b.flag, b.node,
            static_cast<const T *>(b.inl), b.outflow ? static_cast<const T *>(b.ghost[cur]) : nullptr);
        return cudaGetLastError();
    }
    // D3Q19 geometry: the per-site link masks, C := C_b on the inlet nodes of buffer cur and, with
    // an outflow, the ghost column
    static cudaError_t prepare_solid(const Geom &g, const Buffers &b, int cur, int ninl, cudaStream_t st) {
        if (!b.lmask) return cudaErrorInvalidValue;
        k_link_mask<L><<<blocks_for(g.n, 256), 256, 0, st>>>(g, b.node, b.lmask, b.outflow);
        if (ninl > 0)
            k_inlet_fill3<N, T><<<blocks_for(g.n, 256), 256, 0, st>>>(g, b.node, static_cast<const T *>(b.inl),
                                                                      static_cast<T *>(b.C[cur]));
        // column nx - 1 holds no inlet node, so the ghost copy does not race with the fill
        if (b.outflow)
            k_ghost_init<N, T><<<blocks_for((long long)g.ny * g.nz, 256), 256, 0, st>>>(
                g, static_cast<const T *>(b.C[cur]), static_cast<T *>(b.ghost[cur]));
        return cudaGetLastError();
    }
    static cudaError_t inlet_table3(const void *coef, const double *rows, int K, void *out, cudaStream_t st) {
        const Coef<T> &cf = *static_cast<const Coef<T> *>(coef);
        k_inlet_table3<N, T><<<1, kMaxInlets, 0, st>>>(cf, rows, K, static_cast<T *>(out));
        return cudaGetLastError();
    }
    static cudaError_t reduce(const Geom &g, const Buffers &b, int, int nblocks, cudaStream_t st) {
        k_reduce_partial<<<nblocks, 256, 0, st>>>(g.n, N, b.fields, b.partials);
        k_reduce_final<<<1, 256, 0, st>>>(nblocks, N, b.partials, b.flag, b.diag);
        return cudaGetLastError();
    }
    static cudaError_t init_f(const Geom &g, const void *coef, const Buffers &b, int cur, const double *v, cudaStream_t st) {
        const Coef<T> &cf = *static_cast<const Coef<T> *>(coef);
        k_init_f<L, T, SF><<<blocks_for(g.n, 256), 256, 0, st>>>(g, cf, v, static_cast<SF *>(b.f[cur]));
        return cudaGetLastError();
    }
    static cudaError_t unpack_f(const Geom &g, const void *coef, const Buffers &b, int cur, double *out, cudaStream_t st) {
        const Coef<T> &cf = *static_cast<const Coef<T> *>(coef);
        k_unpack_f<L, T, SF><<<blocks_for(g.n, 256), 256, 0, st>>>(g, cf, static_cast<const SF *>(b.f[cur]), out);
        return cudaGetLastError();
    }
    static cudaError_t pack_C(const Geom &g, const Buffers &b, int cur, const double *in, cudaStream_t st) {
        const long long total = g.n * (N - 1);
        k_pack_C<T><<<blocks_for(total, 256), 256, 0, st>>>(total, in, static_cast<T *>(b.C[cur]));
        return cudaGetLastError();
    }
    static cudaError_t init_g(const Geom &g, const void *coef, const Buffers &b, int cur, const double *v, cudaStream_t st) {
        const Coef<T> &cf = *static_cast<const Coef<T> *>(coef);
        k_init_g<L, N, T><<<blocks_for(g.n, 256), 256, 0, st>>>(g, cf, static_cast<const T *>(b.C[cur]), v,
                                                                  static_cast<T *>(b.g[cur]));
        return cudaGetLastError();
    }
};

}  // namespace nfe
