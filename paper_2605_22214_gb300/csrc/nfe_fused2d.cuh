// Fused D2Q9 time step: one kernel per step, one CTA per TX x TY tile.
//
//   phase 1  evolved C on the tile and a 2-site ring -> shared memory (wrapped
//            coordinates), with C_implicit = 1 - sum and the bulk energy E_B
//            (Eq. 5) computed once per site;
//   phase 2  on the tile and a 1-site ring: isotropic grad / Laplacian of every
//            C_i and grad E_B from shared memory (Eqs. 35-36, wall rule of
//            Sec. III C), flux potential S_i = C_i q_i(C) + (3D/4) lap C_i
//            (Eq. 12, factored), force F (Eq. 34), f_k(x) from HBM, v and P
//            (Eqs. 37-38); (C, v, S) of every site -> shared memory;
//   phase 3  tile sites: TRT collision with forcing (Eqs. 23-30), push-stream
//            with halfway bounce-back (Eqs. 44-45);
//   phase 4  tile sites: C_i(x, t+1) = sum_k g^eq_{i,k}(x - e_k) (Eqs. 39-41,
//            tau_g = 1) from the shared (C, v, S) of the 1-ring.
// Only f (8 populations) and the N-1 evolved C are read from and written to
// HBM; every other quantity lives in registers or shared memory.  CTAs whose
// tile plus ring is inside the domain take a path without wrap or wall tests.
// The Cahn-Hilliard gather with bounce-back is chosen from the site's own wall
// mask, never from the tile: its wall-free form is compiled separately, and a
// per-tile choice would let a site's arithmetic depend on the tile shape.
#pragma once

#include "nfe_kernels.cuh"

namespace nfe {

// Shared-memory record of NV values of type T, stored as 16-byte chunks in
// separate planes so that consecutive threads never hit the same bank.
template <typename T, int NV>
struct SRec {
    static constexpr int PER = 16 / sizeof(T);               // values per chunk
    static constexpr int NC = (NV + PER - 1) / PER;           // chunks per record
    static constexpr int NVP = NC * PER;                      // padded count
};

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

template <typename T, int NV>
__device__ __forceinline__ void srec_load(const T *base, int count, int i, T (&out)[SRec<T, NV>::NVP]) {
    using V = typename Vec16<T>::type;
#pragma unroll
    for (int c = 0; c < SRec<T, NV>::NC; ++c) {
        const V v = reinterpret_cast<const V *>(base + size_t(c) * count * SRec<T, NV>::PER)[i];
        if constexpr (sizeof(T) == 4) {
            out[4 * c + 0] = v.x; out[4 * c + 1] = v.y; out[4 * c + 2] = v.z; out[4 * c + 3] = v.w;
        } else {
            out[2 * c + 0] = v.x; out[2 * c + 1] = v.y;
        }
    }
}

template <typename T, int NV>
__device__ __forceinline__ void srec_store(T *base, int count, int i, const T (&in)[SRec<T, NV>::NVP]) {
    using V = typename Vec16<T>::type;
#pragma unroll
    for (int c = 0; c < SRec<T, NV>::NC; ++c) {
        V v;
        if constexpr (sizeof(T) == 4) {
            v.x = in[4 * c + 0]; v.y = in[4 * c + 1]; v.z = in[4 * c + 2]; v.w = in[4 * c + 3];
        } else {
            v.x = in[2 * c + 0]; v.y = in[2 * c + 1];
        }
        reinterpret_cast<V *>(base + size_t(c) * count * SRec<T, NV>::PER)[i] = v;
    }
}

template <int N, typename T, int TX, int TY>
struct Fused2DShape {
    static constexpr int AX = TX + 4, AY = TY + 4, ACOUNT = AX * AY;   // tile + 2-ring
    static constexpr int BX = TX + 2, BY = TY + 2, BCOUNT = BX * BY;   // tile + 1-ring
    using RA = SRec<T, N>;            // evolved C (N-1) and E_B
    using RB = SRec<T, 2 * N>;        // evolved C (N-1), vx, vy, S (N-1)
    static constexpr int A_VALUES = RA::NVP * ACOUNT;
    static constexpr int B_VALUES = RB::NVP * BCOUNT;
    static constexpr size_t BYTES = sizeof(T) * size_t(A_VALUES + B_VALUES);
    static constexpr size_t GEO_BYTES = BYTES + ((ACOUNT + 15) / 16) * 16;   // + node class of tile + 2-ring
    static constexpr int NHALO = BCOUNT - TX * TY;
};

// What the geometry form of the step reads besides the state (all null / 0 without one).
template <typename T>
struct GeoView {
    const unsigned char *node;    // node class per site
    const T *inl;                 // inlet table, 2N values per inlet: vx, vy, C_b (N-1), S_b (N-1)
    const T *ghost;               // outflow ghost column of buffer cur, (N-1) x ny
    int outflow;
};

__device__ __forceinline__ int wrap(int v, int n) {
    // v in [-n, 2n)
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

__device__ __forceinline__ int imod(int v, int n) { return ((v % n) + n) % n; }

// Periodic index of a tile or ring coordinate v in [-2, n + tile + 2): a compare and an add,
// unless the domain is narrower than a tile plus ring (then a full modulo).
__device__ __forceinline__ int pwrap(int v, int n, bool tiny) { return tiny ? imod(v, n) : wrap(v, n); }

// Packed FP32 arithmetic (two values per instruction, sm_100 and later).
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }

// The stencil sums of stencil2d below for FP32, two record values at a time: values 2p and
// 2p + 1 of record A (the evolved C, then E_B) share every instruction.
template <int N, int AX, bool CHECK>
__device__ __forceinline__ void stencil2d_packed(const float *sA, int acount, int ia, unsigned wall,
                                                 float (&c)[N], float (&lap)[N], float (&gx)[N], float (&gy)[N],
                                                 float &gEx, float &gEy) {
    using RA = SRec<float, N>;
    constexpr int NPU = (N + 1) / 2;     // pairs holding the N used values
    float r0[RA::NVP];
    srec_load<float, N>(sA, acount, ia, r0);
    float2 d[9][NPU];
    constexpr int off[9] = {0, 1, -1, AX, -AX, AX + 1, -AX - 1, -AX + 1, AX - 1};
    sfor<1, 9, 1>([&](auto kc_) {
        constexpr int k = decltype(kc_)::value;
        if (CHECK && ((wall >> k) & 1u)) {
#pragma unroll
            for (int p = 0; p < NPU; ++p) d[k][p] = make_float2(0.0f, 0.0f);
        } else {
            float r[RA::NVP];
            srec_load<float, N>(sA, acount, ia + off[k], r);
#pragma unroll
            for (int p = 0; p < NPU; ++p)
                d[k][p] = sub2(make_float2(r[2 * p], r[2 * p + 1]), make_float2(r0[2 * p], r0[2 * p + 1]));
        }
    });
    const float2 third = dup2(1.0f / 3.0f), twelfth = dup2(1.0f / 12.0f), two3 = dup2(2.0f / 3.0f), sixth = dup2(1.0f / 6.0f);
    float L[2 * NPU], X[2 * NPU], Y[2 * NPU];
#pragma unroll
    for (int p = 0; p < NPU; ++p) {
        const float2 ax = add2(add2(d[1][p], d[2][p]), add2(d[3][p], d[4][p]));
        const float2 dg = add2(add2(d[5][p], d[6][p]), add2(d[7][p], d[8][p]));
        const float2 d56 = sub2(d[5][p], d[6][p]), d78 = sub2(d[7][p], d[8][p]);
        const float2 l = fma2(two3, ax, mul2(sixth, dg));                           // (2/c_s^2) sum w_k d_k
        const float2 x = fma2(third, sub2(d[1][p], d[2][p]), mul2(twelfth, add2(d56, d78)));
        const float2 y = fma2(third, sub2(d[3][p], d[4][p]), mul2(twelfth, sub2(d56, d78)));
        L[2 * p] = l.x; L[2 * p + 1] = l.y;
        X[2 * p] = x.x; X[2 * p + 1] = x.y;
        Y[2 * p] = y.x; Y[2 * p + 1] = y.y;
    }
    float sl = 0.0f, sgx = 0.0f, sgy = 0.0f, rest = 0.0f;
#pragma unroll
    for (int a = 0; a < N - 1; ++a) {
        c[a] = r0[a];
        lap[a] = L[a]; gx[a] = X[a]; gy[a] = Y[a];
        sl += L[a]; sgx += X[a]; sgy += Y[a];
        rest += r0[a];
    }
    // implicit component: C_N = 1 - sum, its stencils are minus the sum of the others
    c[N - 1] = 1.0f - rest;
    lap[N - 1] = -sl; gx[N - 1] = -sgx; gy[N - 1] = -sgy;
    gEx = X[N - 1];
    gEy = Y[N - 1];
}

// Stencil of one site from record A at local index ia (row pitch AX).  `wall`
// holds bit k set when x + e_k lies beyond a wall (then that term is dropped).
template <int N, typename T, int AX, bool CHECK>
__device__ __forceinline__ void stencil2d(const T *sA, int acount, int ia, unsigned wall,
                                          T (&c)[N], T (&lap)[N], T (&gx)[N], T (&gy)[N], T &gEx, T &gEy) {
    if constexpr (sizeof(T) == 4) {
        stencil2d_packed<N, AX, CHECK>(sA, acount, ia, wall, c, lap, gx, gy, gEx, gEy);
        return;
    }
    using RA = SRec<T, N>;
    T r0[RA::NVP];
    srec_load<T, N>(sA, acount, ia, r0);
    T d[9][N];            // d[k][a]: neighbour minus centre, a < N-1 volume fractions, a = N-1 bulk energy
    constexpr int off[9] = {0, 1, -1, AX, -AX, AX + 1, -AX - 1, -AX + 1, AX - 1};
    sfor<1, 9, 1>([&](auto kc_) {
        constexpr int k = decltype(kc_)::value;
        if (CHECK && ((wall >> k) & 1u)) {
#pragma unroll
            for (int a = 0; a < N; ++a) d[k][a] = T(0);
        } else {
            T r[RA::NVP];
            srec_load<T, N>(sA, acount, ia + off[k], r);
#pragma unroll
            for (int a = 0; a < N; ++a) d[k][a] = r[a] - r0[a];
        }
    });
    const T third = T(1) / T(3), twelfth = T(1) / T(12), two3 = T(2) / T(3), sixth = T(1) / T(6);
    T sl = T(0), sgx = T(0), sgy = T(0);
#pragma unroll
    for (int a = 0; a < N - 1; ++a) {
        c[a] = r0[a];
        const T ax = (d[1][a] + d[2][a]) + (d[3][a] + d[4][a]);
        const T dg = (d[5][a] + d[6][a]) + (d[7][a] + d[8][a]);
        lap[a] = two3 * ax + sixth * dg;                                    // (2/c_s^2) sum w_k d_k
        gx[a] = third * (d[1][a] - d[2][a]) + twelfth * ((d[5][a] - d[6][a]) + (d[7][a] - d[8][a]));
        gy[a] = third * (d[3][a] - d[4][a]) + twelfth * ((d[5][a] - d[6][a]) - (d[7][a] - d[8][a]));
        sl += lap[a]; sgx += gx[a]; sgy += gy[a];
    }
    // implicit component: C_N = 1 - sum, its stencils are minus the sum of the others
    T rest = T(0);
#pragma unroll
    for (int a = 0; a < N - 1; ++a) rest += r0[a];
    c[N - 1] = T(1) - rest;
    lap[N - 1] = -sl; gx[N - 1] = -sgx; gy[N - 1] = -sgy;
    constexpr int e = N - 1;
    gEx = third * (d[1][e] - d[2][e]) + twelfth * ((d[5][e] - d[6][e]) + (d[7][e] - d[8][e]));
    gEy = third * (d[3][e] - d[4][e]) + twelfth * ((d[5][e] - d[6][e]) - (d[7][e] - d[8][e]));
}

// Phase 2 at one site: S, F, v, P from the stencil and f.  f must hold f_1..f_8.
template <int N, typename T, int Q4>
__device__ __forceinline__ void site_physics(const Coef<T> &cf, const T (&c)[N], const T (&lap)[N],
                                             const T (&gx)[N], const T (&gy)[N], T gEx, T gEy,
                                             const T (&f)[9], T (&S)[N - 1], T &Fx, T &Fy,
                                             T &vx, T &vy, T &P, T &sumf) {
    // force of Eq. 34 (or Eq. 31)
    if (!cf.nonconservative) {
        Fx = gEx; Fy = gEy;
#pragma unroll
        for (int a = 0; a < N; ++a) {
            T h = T(0);
#pragma unroll
            for (int b = 0; b < N; ++b) if (b != a) h += cf.kappa[a][b] * lap[b];
            Fx += h * gx[a]; Fy += h * gy[a];
        }
    } else {
        Fx = T(0); Fy = T(0);
#pragma unroll
        for (int a = 0; a < N; ++a) {
            const T ca = c[a];
            const T fpa = T(2) * ca * (T(1) - T(3) * ca + T(2) * ca * ca);
            T mu = T(0);
#pragma unroll
            for (int b = 0; b < N; ++b) if (b != a) {
                const T t = ca + c[b];
                const T fpt = T(2) * t * (T(1) - T(3) * t + T(2) * t * t);
                mu += cf.beta[a][b] * (fpa - fpt) + cf.kappa[a][b] * lap[b];
            }
            Fx += mu * gx[a]; Fy += mu * gy[a];
        }
    }
    Fx += cf.fb[0]; Fy += cf.fb[1];
    if (cf.has_fc) {
        // body force on one component, F += C_c F_c
        T cc = T(0);
#pragma unroll
        for (int a = 0; a < N; ++a) cc += cf.fcsel[a] * c[a];
        Fx += cc * cf.fc[0]; Fy += cc * cf.fc[1];
    }
    T q[N - 1];
    flux_poly<N, T, Q4>(c, cf, q);
#pragma unroll
    for (int e = 0; e < N - 1; ++e) S[e] = c[e] * q[e] + cf.d34 * lap[e];
    flux_rest<N, T, Q4>(c, cf, S);
    // moments (Eqs. 37-38), rho = 1
    const T jx = (f[1] - f[2]) + (f[5] - f[6]) + (f[7] - f[8]);
    const T jy = (f[3] - f[4]) + (f[5] - f[6]) - (f[7] - f[8]);
    sumf = ((f[1] + f[2]) + (f[3] + f[4])) + ((f[5] + f[6]) + (f[7] + f[8]));
    vx = jx + T(0.5) * Fx;
    vy = jy + T(0.5) * Fy;
    const T w0 = T(4) / T(9);
    P = (sumf - T(1.5) * w0 * (vx * vx + vy * vy)) * T(1.0 / (3.0 * (1.0 - 4.0 / 9.0)));
}

// One tile of the fused step (phases 1-4 above).  `smem` holds
// Fused2DShape<N, T, TX, TY>::BYTES bytes; all TX * TY threads of the CTA call it.
// Global loads of the step's inputs: plain, or L2-only (ld.global.cg) when the
// inputs were written earlier in the same launch by other CTAs.
template <bool L2ONLY, typename X>
__device__ __forceinline__ X ldin(const X *p) {
    if constexpr (L2ONLY) return __ldcg(p);
    else return *p;
}

template <bool L2ONLY, typename SF, typename T>
__device__ __forceinline__ T fload(const SF *p, double w, T finv) {
    if constexpr (L2ONLY) {
        static_assert(sizeof(SF) >= 4, "L2-only loads are used with FP32 / FP64 storage");
        return T(__ldcg(p));
    } else {
        return FStore<SF, T>::load(p, w, finv);
    }
}

// TAUG: the stored-g path (tau_g != 1), with the component populations in gin / gout.
// GEO: node classes (solid nodes, inlets, outflow ghost column) from `geo`; see the boundary
// rules at the phases below.
// CSYNC: cf is being copied into shared memory by the caller while the tile starts; the tile
// issues its f and C loads first and reads cf only after a block barrier.
template <int N, typename T, typename SF, int TX, int TY, bool L2ONLY, int Q4, bool TAUG = false, bool GEO = false,
          bool CSYNC = false>
__device__ __forceinline__ void fused2d_tile(const Geom &g, const Coef<T> &cf, const SF *__restrict__ fin,
                                             SF *__restrict__ fout, const T *__restrict__ Cin,
                                             T *__restrict__ Cout, int *__restrict__ flag,
                                             int x0, int y0, unsigned char *smem,
                                             const T *__restrict__ gin = nullptr, T *__restrict__ gout = nullptr,
                                             GeoView<T> geo = {}) {
    using Sh = Fused2DShape<N, T, TX, TY>;
    using RA = typename Sh::RA;
    using RB = typename Sh::RB;
    static_assert(Sh::NHALO <= TX * TY, "one ring site per thread at most");
    T *sA = reinterpret_cast<T *>(smem);
    T *sB = sA + Sh::A_VALUES;
    unsigned char *sN = reinterpret_cast<unsigned char *>(sB + Sh::B_VALUES);   // GEO only
    const int nx = g.nx, ny = g.ny;
    const int n = int(g.n);
    const int tid = threadIdx.x;
    // uniform per CTA: does the tile plus its 2-ring cross the domain edge (indices wrap or
    // clamp), is that edge a wall (stencils need wall tests), is the domain narrower than a tile?
    const bool edge = (x0 - 2 < 0) || (x0 + TX + 2 > nx) || (y0 - 2 < 0) || (y0 + TY + 2 > ny);
    const bool wallt = (g.wx && ((x0 - 2 < 0) || (x0 + TX + 2 > nx))) || (g.wy && ((y0 - 2 < 0) || (y0 + TY + 2 > ny)));
    const bool tiny = nx < TX + 4 || ny < TY + 4;

    // ---- own site and ring site of this thread; start their f loads first ----
    const int tx = tid % TX, ty = tid / TX;
    const int gx0 = x0 + tx, gy0 = y0 + ty;
    const bool own = gx0 < nx && gy0 < ny;             // ragged far edge: duplicates only
    const int sx = edge ? pwrap(gx0, nx, tiny) : gx0;  // wrapped (periodic duplicates)
    const int sy = edge ? pwrap(gy0, ny, tiny) : gy0;
    const int s0 = sx + nx * sy;
    T f[9];
    f[0] = T(0);
    sfor<1, 9, 1>([&](auto kc_) { constexpr int k = decltype(kc_)::value; f[k] = fload<L2ONLY, SF, T>(fin + (k - 1) * n + s0, LD2Q9::w(k), cf.finv); });

    // ring of the tile+1 region: top row, bottom row, then left and right columns
    int bx = 0, by = 0;
    const bool has_ring = tid < Sh::NHALO;
    if (tid < Sh::BX) { bx = tid; by = 0; }
    else if (tid < 2 * Sh::BX) { bx = tid - Sh::BX; by = Sh::BY - 1; }
    else { const int r = tid - 2 * Sh::BX; by = 1 + (r >> 1); bx = (r & 1) ? Sh::BX - 1 : 0; }
    const int hx = x0 + bx - 1, hy = y0 + by - 1;
    bool ring_ok = has_ring;
    unsigned hwall = 0;
    int hs = hx + nx * hy;
    if (edge && has_ring) {
        if ((g.wx && (hx < 0 || hx >= nx)) || (g.wy && (hy < 0 || hy >= ny))) ring_ok = false;
        hs = pwrap(hx, nx, tiny) + nx * pwrap(hy, ny, tiny);
    }
    if (!GEO && wallt && has_ring) {
        sfor<1, 9, 1>([&](auto kc_) {
            constexpr int k = decltype(kc_)::value;
            const int xx = hx + LD2Q9::ex(k), yy = hy + LD2Q9::ey(k);
            if ((g.wx && (xx < 0 || xx >= nx)) || (g.wy && (yy < 0 || yy >= ny))) hwall |= 1u << k;
        });
    }
    T hf[9];
    hf[0] = T(0);
    if (ring_ok) {
        sfor<1, 9, 1>([&](auto kc_) { constexpr int k = decltype(kc_)::value; hf[k] = fload<L2ONLY, SF, T>(fin + (k - 1) * n + hs, LD2Q9::w(k), cf.finv); });
    }

    // ---- phase 1: C and E_B on tile + 2-ring ---------------------------------
    // every load of the phase is issued before any of them is used (plain loads into registers:
    // staging them by cp.async and completing E_B from shared memory measured 5 % slower, the
    // tile being loaded once per CTA with nothing to overlap the copies with)
    constexpr int NT = TX * TY;
    constexpr int ITER = (Sh::ACOUNT + NT - 1) / NT;
    T cl[ITER][N - 1];
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int i = tid + it * NT;
        if (i < Sh::ACOUNT) {
            const int ly = i / Sh::AX, lx = i - ly * Sh::AX;
            const int gxu = x0 + lx - 2, gyu = y0 + ly - 2;
            int gx = gxu, gy = gyu;
            if (edge) {
                // periodic wrap; beyond a wall (or a ragged far edge) clamp to a real site:
                // such entries are never used by a real site's stencil
                gx = g.wx ? min(max(gx, 0), nx - 1) : pwrap(gx, nx, tiny);
                gy = g.wy ? min(max(gy, 0), ny - 1) : pwrap(gy, ny, tiny);
            }
            const int s = gx + nx * gy;
            if constexpr (GEO) {
                // beyond the outflow edge: the ghost column (its class that of column nx - 1,
                // ghost where that is not solid); beyond an edge wall: solid
                const bool gcol = geo.outflow && gxu >= nx;
                if (gcol) {
#pragma unroll
                    for (int a = 0; a < N - 1; ++a) cl[it][a] = geo.ghost[a * ny + gy];
                } else {
#pragma unroll
                    for (int a = 0; a < N - 1; ++a) cl[it][a] = ldin<L2ONLY>(Cin + a * n + s);
                }
                unsigned char cls;
                if ((g.wx && (gxu < 0 || gxu >= nx)) || (g.wy && (gyu < 0 || gyu >= ny))) cls = kNodeSolid;
                else if (gcol) cls = geo.node[(nx - 1) + nx * gy] == kNodeSolid ? kNodeSolid : kNodeGhost;
                else cls = geo.node[s];
                sN[i] = cls;
            } else {
#pragma unroll
                for (int a = 0; a < N - 1; ++a) cl[it][a] = ldin<L2ONLY>(Cin + a * n + s);
            }
        }
    }
    if constexpr (CSYNC) __syncthreads();      // the caller's copy of cf is complete
#pragma unroll
    for (int it = 0; it < ITER; ++it) {
        const int i = tid + it * NT;
        if (i < Sh::ACOUNT) {
            T rec[RA::NVP];
            T cc[N];
            T rest = T(0);
#pragma unroll
            for (int a = 0; a < N - 1; ++a) { cc[a] = cl[it][a]; rec[a] = cc[a]; rest += cc[a]; }
            cc[N - 1] = T(1) - rest;
            rec[N - 1] = bulk_energy<N, T>(cc, cf);
#pragma unroll
            for (int a = N; a < RA::NVP; ++a) rec[a] = T(0);
            srec_store<T, N>(sA, Sh::ACOUNT, i, rec);
        }
    }
    __syncthreads();

    // ---- phase 2a: own site ---------------------------------------------------
    // wall mask of the own site: bit k set when x + e_k is beyond a wall
    // GEO: wall0 = solid neighbours (mirror rule, bounce-back), open0 = every non-fluid
    // neighbour (inlet, solid, ghost: no plain push there), cls0 = the site's own class
    unsigned wall0 = 0, open0 = 0;
    unsigned char cls0 = kNodeFluid;
    if constexpr (GEO) {
        const int ia = (ty + 2) * Sh::AX + (tx + 2);
        cls0 = sN[ia];
        sfor<1, 9, 1>([&](auto kc_) {
            constexpr int k = decltype(kc_)::value;
            const unsigned char cl = sN[ia + LD2Q9::ex(k) + Sh::AX * LD2Q9::ey(k)];
            if (cl == kNodeSolid) wall0 |= 1u << k;
            if (cl != kNodeFluid) open0 |= 1u << k;
        });
    } else if (wallt) {
        sfor<1, 9, 1>([&](auto kc_) {
            constexpr int k = decltype(kc_)::value;
            const int xx = gx0 + LD2Q9::ex(k), yy = gy0 + LD2Q9::ey(k);
            if ((g.wx && (xx < 0 || xx >= nx)) || (g.wy && (yy < 0 || yy >= ny))) wall0 |= 1u << k;
        });
    }
    T c[N], lap[N], gxv[N], gyv[N], gEx, gEy;
    T S[N - 1], Fx, Fy, vx, vy, P, sumf;
    {
        const int ia = (ty + 2) * Sh::AX + (tx + 2);
        // GEO: one choice per warp (the checked form gives the same values where no neighbour is
        // solid, and a per-site choice would run both forms in every warp that meets a post)
        if (GEO ? __any_sync(0xffffffffu, wall0 != 0u) : wallt)
            stencil2d<N, T, Sh::AX, true>(sA, Sh::ACOUNT, ia, wall0, c, lap, gxv, gyv, gEx, gEy);
        else
            stencil2d<N, T, Sh::AX, false>(sA, Sh::ACOUNT, ia, 0u, c, lap, gxv, gyv, gEx, gEy);
        site_physics<N, T, Q4>(cf, c, lap, gxv, gyv, gEx, gEy, f, S, Fx, Fy, vx, vy, P, sumf);
        if constexpr (GEO) {
            // an inlet node's record is its prescribed state (C_b is its stored C)
            if (cls0 >= kNodeInlet0 && cls0 != kNodeGhost) {
                const T *row = geo.inl + (cls0 - kNodeInlet0) * (2 * N);
                vx = row[0]; vy = row[1];
#pragma unroll
                for (int a = 0; a < N - 1; ++a) S[a] = row[N + 1 + a];
            }
        }
        T rec[RB::NVP];
#pragma unroll
        for (int a = 0; a < N - 1; ++a) { rec[a] = c[a]; rec[N + 1 + a] = S[a]; }
        rec[N - 1] = vx; rec[N] = vy;
#pragma unroll
        for (int a = 2 * N; a < RB::NVP; ++a) rec[a] = T(0);
        srec_store<T, 2 * N>(sB, Sh::BCOUNT, (ty + 1) * Sh::BX + (tx + 1), rec);
    }

    // ---- phase 2b: the 1-ring around the tile (sites beyond a wall are skipped:
    //      sources there are replaced by bounce-back) ---------------------------
    if (ring_ok) {
        T hc[N], hl[N], hgx[N], hgy[N], hEx, hEy;
        const int ia = (by + 1) * Sh::AX + (bx + 1);
        unsigned char hcls = kNodeFluid;
        if constexpr (GEO) {
            hcls = sN[ia];
            sfor<1, 9, 1>([&](auto kc_) {
                constexpr int k = decltype(kc_)::value;
                if (sN[ia + LD2Q9::ex(k) + Sh::AX * LD2Q9::ey(k)] == kNodeSolid) hwall |= 1u << k;
            });
        }
        if (GEO ? __any_sync(__activemask(), hwall != 0u) : wallt)
            stencil2d<N, T, Sh::AX, true>(sA, Sh::ACOUNT, ia, hwall, hc, hl, hgx, hgy, hEx, hEy);
        else
            stencil2d<N, T, Sh::AX, false>(sA, Sh::ACOUNT, ia, 0u, hc, hl, hgx, hgy, hEx, hEy);
        T hS[N - 1], hFx, hFy, hvx, hvy, hP, hsum;
        site_physics<N, T, Q4>(cf, hc, hl, hgx, hgy, hEx, hEy, hf, hS, hFx, hFy, hvx, hvy, hP, hsum);
        if constexpr (GEO) {
            if (hcls >= kNodeInlet0 && hcls != kNodeGhost) {
                const T *row = geo.inl + (hcls - kNodeInlet0) * (2 * N);
                hvx = row[0]; hvy = row[1];
#pragma unroll
                for (int a = 0; a < N - 1; ++a) hS[a] = row[N + 1 + a];
            }
        }
        T rec[RB::NVP];
#pragma unroll
        for (int a = 0; a < N - 1; ++a) { rec[a] = hc[a]; rec[N + 1 + a] = hS[a]; }
        rec[N - 1] = hvx; rec[N] = hvy;
#pragma unroll
        for (int a = 2 * N; a < RB::NVP; ++a) rec[a] = T(0);
        srec_store<T, 2 * N>(sB, Sh::BCOUNT, by * Sh::BX + bx, rec);
    }

    // ---- phase 3: collide and push-stream the own site ----------------------
    // GEO: a non-fluid node keeps its populations (copied bit for bit to the new buffer)
    if (GEO && own && cls0 != kNodeFluid) {
#pragma unroll
        for (int k = 1; k < 9; ++k) fout[(k - 1) * n + s0] = fin[(k - 1) * n + s0];
    }
    if (own && (!GEO || cls0 == kNodeFluid)) {
        T op, om;
        relaxation<N, T>(cf, c, op, om);
        const T ap = T(1) - T(0.5) * op, am = T(1) - T(0.5) * om;
        const T vv = vx * vx + vy * vy, vF = vx * Fx + vy * Fy;
        const T base = T(3) * P - T(1.5) * vv;
        // TRT with forcing (Eqs. 23-30) regrouped so that per-site factors are formed once:
        // for a pair (k, kbar), with s = f_k + f_kbar and d = f_k - f_kbar,
        //   sym  = w_k [X + e.v (Y e.v + Z e.F)] - (op / 2) s
        //   anti = w_k (U e.v + V e.F) - (om / 2) d
        // where X = op (3P - 1.5 v.v) - 3 ap v.F, Y = 4.5 op, Z = 9 ap, U = 3 om, V = 3 am;
        // w_k X ... w_k V are shared by all pairs of one weight class.
        const T hop = T(0.5) * op, hom = T(0.5) * om;
        const T X = op * base - T(3) * ap * vF, Y = T(4.5) * op, Z = T(9) * ap, U = T(3) * om, V = T(3) * am;
        // GEO: plain neighbour offsets for a site inside the domain by one site with only fluid
        // neighbours (the general store block gives the same stores there; one choice per warp).
        // Otherwise every site without an adjacent wall takes one store sequence with the periodic
        // wrap folded into its neighbour offsets, so the sites of a warp do not diverge at the edges.
        bool fast;
        if constexpr (GEO) fast = __all_sync(__activemask(), sx > 0 && sx < nx - 1 && sy > 0 && sy < ny - 1 && open0 == 0u);
        else fast = wall0 == 0u;
        if constexpr (sizeof(T) == 4) {
            // FP32: the two pairs of one weight class share every instruction, pair (1, 2) or
            // (5, 6) in the first lane and (3, 4) or (7, 8) in the second
            const float2 mhop = dup2(-hop), mhom = dup2(-hom);
            auto cls = [&](float wk, float2 eu, float2 eF, float &fa, float &fab, float &fc, float &fcb) {
                const float2 fk = make_float2(fa, fc), fkb = make_float2(fab, fcb);
                const float2 sp = add2(fk, fkb), dm = sub2(fk, fkb);
                const float2 sym = fma2(mhop, sp, fma2(eu, fma2(dup2(wk * Y), eu, mul2(dup2(wk * Z), eF)), dup2(wk * X)));
                const float2 anti = fma2(mhom, dm, fma2(dup2(wk * U), eu, mul2(dup2(wk * V), eF)));
                const float2 pk = add2(fk, add2(sym, anti)), pkb = add2(fkb, sub2(sym, anti));
                fa = pk.x; fc = pk.y; fab = pkb.x; fcb = pkb.y;
            };
            cls(float(LD2Q9::w(1)), make_float2(vx, vy), make_float2(Fx, Fy), f[1], f[2], f[3], f[4]);
            cls(float(LD2Q9::w(5)), make_float2(vx + vy, vx - vy), make_float2(Fx + Fy, Fx - Fy), f[5], f[6], f[7], f[8]);
        } else {
        sfor<1, 9, 2>([&](auto kc_) {
            constexpr int k = decltype(kc_)::value;
            const int kb = k + 1;
            const T wk = T(LD2Q9::w(k));
            const T eu = T(LD2Q9::ex(k)) * vx + T(LD2Q9::ey(k)) * vy;
            const T eF = T(LD2Q9::ex(k)) * Fx + T(LD2Q9::ey(k)) * Fy;
            const T sp = f[k] + f[kb], dm = f[k] - f[kb];
            const T sym = (wk * X + eu * ((wk * Y) * eu + (wk * Z) * eF)) - hop * sp;
            const T anti = ((wk * U) * eu + (wk * V) * eF) - hom * dm;
            // post-collision values replace f in place (each pair is read once)
            f[k] = f[k] + sym + anti;
            f[kb] = f[kb] + sym - anti;
        });
        }
        // one branch around the whole store block: inside the unrolled loop the compiler
        // would predicate both forms for every site
        if (fast) {
            if constexpr (GEO) {
                sfor<1, 9, 1>([&](auto kc_) {
                    constexpr int k = decltype(kc_)::value;
                    constexpr int dk0 = LD2Q9::ex(k);
                    const int dk = dk0 + nx * LD2Q9::ey(k);
                    FStore<SF, T>::store(fout + (k - 1) * n + (s0 + dk), f[k], LD2Q9::w(k), cf.fscale);
                });
            } else {
                const int dxp = sx == nx - 1 ? 1 - nx : 1, dxm = sx == 0 ? nx - 1 : -1;
                const int dyp = sy == ny - 1 ? nx - n : nx, dym = sy == 0 ? n - nx : -nx;
                sfor<1, 9, 1>([&](auto kc_) {
                    constexpr int k = decltype(kc_)::value;
                    constexpr int ex = LD2Q9::ex(k), ey = LD2Q9::ey(k);
                    int t = s0;
                    if constexpr (ex != 0) t += ex > 0 ? dxp : dxm;
                    if constexpr (ey != 0) t += ey > 0 ? dyp : dym;
                    FStore<SF, T>::store(fout + (k - 1) * n + t, f[k], LD2Q9::w(k), cf.fscale);
                });
            }
        } else if constexpr (GEO) {
            const int ia = (ty + 2) * Sh::AX + (tx + 2);
            sfor<1, 9, 1>([&](auto kc_) {
                constexpr int k = decltype(kc_)::value;
                constexpr int kb = opp(k);
                const unsigned char cl = sN[ia + LD2Q9::ex(k) + Sh::AX * LD2Q9::ey(k)];
                if (cl == kNodeFluid) {
                    FStore<SF, T>::store(fout + (k - 1) * n + (wrap(sx + LD2Q9::ex(k), nx) + nx * wrap(sy + LD2Q9::ey(k), ny)),
                                         f[k], LD2Q9::w(k), cf.fscale);
                } else if (cl == kNodeSolid) {
                    FStore<SF, T>::store(fout + (kb - 1) * n + s0, f[k], LD2Q9::w(kb), cf.fscale);
                } else if (cl != kNodeGhost) {
                    // inlet j (moving-wall bounce-back, rho_b = 1):
                    // f_kbar(x, t+1) = post_k(x) - 2 w_k (e_k . v_b) / c_s^2
                    const T *row = geo.inl + (cl - kNodeInlet0) * (2 * N);
                    const T ev = T(LD2Q9::ex(k)) * row[0] + T(LD2Q9::ey(k)) * row[1];
                    FStore<SF, T>::store(fout + (kb - 1) * n + s0, f[k] - T(6.0 * LD2Q9::w(k)) * ev, LD2Q9::w(kb), cf.fscale);
                }
                // into the ghost column: the population leaves the domain
            });
        } else {
            sfor<1, 9, 1>([&](auto kc_) {
                constexpr int k = decltype(kc_)::value;
                constexpr int kb = opp(k);
                // halfway bounce-back: f_kbar(x, t+1) = post_k(x)
                if ((wall0 >> k) & 1u) FStore<SF, T>::store(fout + (kb - 1) * n + s0, f[k], LD2Q9::w(kb), cf.fscale);
                else FStore<SF, T>::store(fout + (k - 1) * n + (wrap(sx + LD2Q9::ex(k), nx) + nx * wrap(sy + LD2Q9::ey(k), ny)),
                                          f[k], LD2Q9::w(k), cf.fscale);
            });
        }
    }
    __syncthreads();

    // ---- phase 4 with stored g (tau_g != 1): pull, relax and bounce back -----
    // g_k(x, t+1) = g*_k(x - e_k), g* = g + (g^eq - g) / tau_g, with g^eq_k(x - e_k) from the
    // shared (C, v, S) records; a source beyond a wall gives g*_kbar(x) (Eqs. 44-45); then
    // C_i(x, t+1) = sum_k g_{i,k}(x, t+1) (Eq. 41).
    if constexpr (TAUG) {
        if (own) {
            const T m = cf.m, omg = cf.gomega;
            const int ib = (ty + 1) * Sh::BX + (tx + 1);
            T r0[RB::NVP];
            srec_load<T, 2 * N>(sB, Sh::BCOUNT, ib, r0);
            const T vv0 = r0[N - 1] * r0[N - 1] + r0[N] * r0[N];
            const bool fast = sx > 0 && sx < nx - 1 && sy > 0 && sy < ny - 1;
            constexpr int offB[9] = {0, 1, -1, TX + 2, -(TX + 2), TX + 3, -(TX + 3), -(TX + 2) + 1, (TX + 2) - 1};
            constexpr int Q = 9;
            T csum[N - 1];
#pragma unroll
            for (int e = 0; e < N - 1; ++e) csum[e] = T(0);
            sfor<0, 9, 1>([&](auto kc_) {
                constexpr int k = decltype(kc_)::value;
                const T wk = T(LD2Q9::w(k));
                if constexpr (k == 0) {
                    const T s0k = wk * (-T(1.5) * vv0);
#pragma unroll
                    for (int e = 0; e < N - 1; ++e) {
                        const T geq = r0[e] * (T(1) + s0k) + (T(1) - wk) * m * r0[N + 1 + e];
                        const T gg = gin[size_t(e * Q) * n + s0];
                        const T post = gg + omg * (geq - gg);
                        gout[size_t(e * Q) * n + s0] = post;
                        csum[e] += post;
                    }
                } else {
                    constexpr int kb = opp(k);
                    if (wall0 && ((wall0 >> kb) & 1u)) {
                        const T eu = T(LD2Q9::ex(kb)) * r0[N - 1] + T(LD2Q9::ey(kb)) * r0[N];
                        const T skb = wk * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * vv0);
#pragma unroll
                        for (int e = 0; e < N - 1; ++e) {
                            const T geq = r0[e] * skb - wk * m * r0[N + 1 + e];
                            const T gg = gin[size_t(e * Q + kb) * n + s0];
                            const T post = gg + omg * (geq - gg);
                            gout[size_t(e * Q + k) * n + s0] = post;
                            csum[e] += post;
                        }
                    } else {
                        T r[RB::NVP];
                        srec_load<T, 2 * N>(sB, Sh::BCOUNT, ib + offB[kb], r);
                        const T eu = T(LD2Q9::ex(k)) * r[N - 1] + T(LD2Q9::ey(k)) * r[N];
                        const T sk = wk * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * (r[N - 1] * r[N - 1] + r[N] * r[N]));
                        const int src = fast ? s0 - (LD2Q9::ex(k) + nx * LD2Q9::ey(k))
                                             : wrap(sx - LD2Q9::ex(k), nx) + nx * wrap(sy - LD2Q9::ey(k), ny);
#pragma unroll
                        for (int e = 0; e < N - 1; ++e) {
                            const T geq = r[e] * sk - wk * m * r[N + 1 + e];
                            const T gg = gin[size_t(e * Q + k) * n + src];
                            const T post = gg + omg * (geq - gg);
                            gout[size_t(e * Q + k) * n + s0] = post;
                            csum[e] += post;
                        }
                    }
                }
            });
            bool bad = false;
#pragma unroll
            for (int e = 0; e < N - 1; ++e) {
                Cout[e * n + s0] = csum[e];
                bad |= !isfinite(csum[e]);
            }
            if (bad) atomicOr(flag, 1);
        }
        return;
    }

    // ---- phase 4: Cahn-Hilliard update of the own site ----------------------
    // GEO: a non-fluid node keeps its volume fractions; links from an inlet node carry the
    // equilibrium of its prescribed record, links from a solid node bounce back (wall0)
    if (GEO && own && cls0 != kNodeFluid) {
#pragma unroll
        for (int e = 0; e < N - 1; ++e) Cout[e * n + s0] = Cin[e * n + s0];
    }
    if (own && (!GEO || cls0 == kNodeFluid)) {
        const T m = cf.m;
        const T w0 = T(4) / T(9);
        const int ib = (ty + 1) * Sh::BX + (tx + 1);
        T r0[RB::NVP];
        srec_load<T, 2 * N>(sB, Sh::BCOUNT, ib, r0);
        const T vv0 = r0[N - 1] * r0[N - 1] + r0[N] * r0[N];
        T acc[N - 1], lapS[N - 1];
#pragma unroll
        // acc gathers only the small advective increments; C(x) is added once at the end, so in
        // FP32 the rest-population share C s_0 is not lost against 1 (mass-exact update)
        for (int e = 0; e < N - 1; ++e) { acc[e] = r0[e] * (-T(1.5) * w0 * vv0); lapS[e] = T(0); }
        constexpr int offB[9] = {0, 1, -1, TX + 2, -(TX + 2), TX + 3, -(TX + 3), -(TX + 2) + 1, (TX + 2) - 1};
        // the wall-free form carries no bounce-back code (no predicated second path)
        auto gather = [&](auto chk_) {
            constexpr bool CHECK = decltype(chk_)::value;
            sfor<1, 9, 1>([&](auto kc_) {
                constexpr int k = decltype(kc_)::value;
                const T wk = T(LD2Q9::w(k));
                // source x - e_k is the neighbour in direction kbar
                const int kb = opp(k);
                if (CHECK && ((wall0 >> kb) & 1u)) {
                    // bounce-back: g_k(x, t+1) = g^eq_kbar(x, t); its S difference is zero
                    const T eu = -(T(LD2Q9::ex(k)) * r0[N - 1] + T(LD2Q9::ey(k)) * r0[N]);
                    const T sk = wk * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * vv0);
#pragma unroll
                    for (int e = 0; e < N - 1; ++e) acc[e] += r0[e] * sk;
                } else {
                    T r[RB::NVP];
                    srec_load<T, 2 * N>(sB, Sh::BCOUNT, ib + offB[kb], r);
                    const T eu = T(LD2Q9::ex(k)) * r[N - 1] + T(LD2Q9::ey(k)) * r[N];
                    const T sk = wk * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * (r[N - 1] * r[N - 1] + r[N] * r[N]));
#pragma unroll
                    for (int e = 0; e < N - 1; ++e) { acc[e] += r[e] * sk; lapS[e] += wk * (r[N + 1 + e] - r0[N + 1 + e]); }
                }
            });
        };
        // decided per site (not per tile), so a site runs the same code under every tile shape;
        // the geometry form (one tile shape) decides per warp, the checked form giving the same
        // values where no neighbour is solid
        if (GEO ? __any_sync(__activemask(), wall0 != 0u) : wall0 != 0u) gather(std::true_type{});
        else gather(std::false_type{});
        bool bad = false;
#pragma unroll
        for (int e = 0; e < N - 1; ++e) {
            // m [(1 - w_0) S(x) - sum_k w_k S(x - e_k)] written as differences: every link's
            // two contributions are exact negatives, so the FP32 update conserves mass
            const T out = r0[e] + (acc[e] - m * lapS[e]);
            Cout[e * n + s0] = out;
            bad |= !isfinite(out);
        }
        if (bad) atomicOr(flag, 1);
    }
}

// Minimum resident CTAs per SM requested from the register allocator.  The FP32 tile shapes
// get different budgets (32x4 and 32x16: 64 registers; 32x8: 85, three CTAs per SM) and the
// autotuner times them all, so each workload runs the trade-off of spills against occupancy
// that suits it.
template <typename T, int NT> struct Fused2DOcc { static constexpr int value = sizeof(T) == 4 ? (NT <= 128 ? 8 : NT <= 256 ? 3 : 2) : 1; };

template <int N, typename T, typename SF, int TX, int TY, int Q4, bool TAUG, bool GEO = false>
__global__ void __launch_bounds__(TX * TY, (Fused2DOcc<T, TX * TY>::value))
k_fused2d(Geom g, Coef<T> cf, const SF *__restrict__ fin, SF *__restrict__ fout,
          const T *__restrict__ Cin, T *__restrict__ Cout, int *__restrict__ flag,
          const T *__restrict__ gin, T *__restrict__ gout, GeoView<T> geo) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fused2d_tile<N, T, SF, TX, TY, false, Q4, TAUG, GEO>(g, cf, fin, fout, Cin, Cout, flag, blockIdx.x * TX,
                                                         blockIdx.y * TY, smem_raw, gin, gout, geo);
}

template <int N, typename T, typename SF, int TX, int TY, int Q4, bool TAUG = false, bool GEO = false>
cudaError_t launch_fused2d(const Geom &g, const Coef<T> &cf, const Buffers &b, int cur, cudaStream_t st) {
    using Sh = Fused2DShape<N, T, TX, TY>;
    constexpr size_t bytes = GEO ? Sh::GEO_BYTES : Sh::BYTES;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_fused2d<N, T, SF, TX, TY, Q4, TAUG, GEO>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    const dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY);
    GeoView<T> geo{};
    if constexpr (GEO) geo = {b.node, static_cast<const T *>(b.inl), static_cast<const T *>(b.ghost[cur]), b.outflow};
    k_fused2d<N, T, SF, TX, TY, Q4, TAUG, GEO><<<grid, TX * TY, bytes, st>>>(
        g, cf, static_cast<const SF *>(b.f[cur]), static_cast<SF *>(b.f[1 - cur]),
        static_cast<const T *>(b.C[cur]), static_cast<T *>(b.C[1 - cur]), b.flag,
        static_cast<const T *>(b.g[cur]), static_cast<T *>(b.g[1 - cur]), geo);
    return cudaGetLastError();
}

}  // namespace nfe

#include "nfe_geo2d.cuh"

namespace nfe {

// D2Q9 dispatch: the fused step with three tile heights (TX = 32).
template <int N, typename T, typename SF>
struct Fused2DLaunch {
    static cudaError_t step(const Geom &g, const void *coef, const Buffers &b, int cur, cudaStream_t st, int variant) {
        const Coef<T> &cf = *static_cast<const Coef<T> *>(coef);
        // stored g (tau_g != 1): one tile shape
        if (b.g[0]) return launch_fused2d<N, T, SF, 32, 8, Q4_GLOBAL, true>(g, cf, b, cur, st);
        // open and complex boundaries: one tile shape, then the convective outflow
        if (b.node) {
            cudaError_t e = launch_fused2d<N, T, SF, 32, 8, Q4_GLOBAL, false, true>(g, cf, b, cur, st);
            if (e == cudaSuccess && b.outflow) e = launch_outflow2d<N, T, SF>(g, cf, b, cur, st);
            return e;
        }
        if (cf.no_phi) return launch<Q4_NOPHI>(g, cf, b, cur, st, variant);
        return cf.has_q4 ? launch<Q4_GLOBAL>(g, cf, b, cur, st, variant) : launch<Q4_ABSENT>(g, cf, b, cur, st, variant);
    }
    template <int Q4>
    static cudaError_t launch(const Geom &g, const Coef<T> &cf, const Buffers &b, int cur, cudaStream_t st, int variant) {
        switch (variant) {
            case 0: return launch_fused2d<N, T, SF, 32, 4, Q4>(g, cf, b, cur, st);
            case 1: return launch_fused2d<N, T, SF, 32, 8, Q4>(g, cf, b, cur, st);
            default: return launch_fused2d<N, T, SF, 32, 16, Q4>(g, cf, b, cur, st);
        }
    }
    static const Ops *ops(int prec) {
        using B = Launch<LD2Q9, N, T, SF>;
        static const Ops o = {9, 2, N, prec, 1, {K_FUSED, K_FUSED}, {&step, nullptr}, 3,
                              {"fused 32x4", "fused 32x8", "fused 32x16", nullptr},
                              &B::moments, &B::reduce, &B::init_f, &B::unpack_f, &B::pack_C, &B::init_g,
                              int(sizeof(SF)), int(sizeof(T)),
                              &GeoOps<N, T, SF>::inlet_table, &GeoOps<N, T, SF>::prepare, &GeoOps<N, T, SF>::moments};
        return &o;
    }
};

// N = 2 .. 4 and N = 5 .. 8 are instantiated in separate translation units (compiled in parallel).
template <typename T, typename SF>
const Ops *ops_fused2d_lo(int N, int prec) {
    switch (N) {
        case 2: return Fused2DLaunch<2, T, SF>::ops(prec);
        case 3: return Fused2DLaunch<3, T, SF>::ops(prec);
        case 4: return Fused2DLaunch<4, T, SF>::ops(prec);
        default: return nullptr;
    }
}

// One component count per call (the N = 5..8 translation units instantiate two counts each).
template <int NN, typename T, typename SF>
const Ops *ops_fused2d_one(int prec) { return Fused2DLaunch<NN, T, SF>::ops(prec); }

}  // namespace nfe
