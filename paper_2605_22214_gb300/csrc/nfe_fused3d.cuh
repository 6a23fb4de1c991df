// Fused D3Q19 time step: one kernel per step.  A CTA owns a TX x TY column of
// the grid over a chunk of z-planes and marches up in z with shared-memory
// ring buffers:
//   A ring (4 planes, tile + 2-site ring in x/y): evolved C, staged from HBM by
//     cp.async two planes ahead of use, and the bulk energy E_B (Eq. 5) computed
//     once per site from the staged values;
//   B ring (3 planes, tile + 1-site ring): evolved C, v, the flux potential S and |v|^2.
// For every plane z of the chunk the CTA
//   1. completes A-plane z+2 (its cp.async copies, then E_B),
//   2. computes B-plane z+1: isotropic grad / Laplacian (Eqs. 35-36) from A-planes
//      z..z+2, S_i = C_i q_i(C) + (3D/4) lap C_i (Eq. 12), the force of Eq. 34,
//      moments of f (Eqs. 37-38); the own sites of plane z+1 are collided (TRT with
//      forcing, Eqs. 23-30) and push-streamed with bounce-back (Eqs. 44-45),
//   3. starts the copies of A-plane z+3 and the loads of the populations of plane z+2,
//   4. computes C(t+1) of plane z from B-planes z-1..z+1 (Eqs. 39-41, tau_g = 1).
// Only f (18 populations) and the N-1 evolved C cross HBM; the redundant work is
// the x/y ring only, the z direction is streamed.
//
// In FP32 the stencil sums, the moments, the collision and the Cahn-Hilliard gather run on
// packed FP32x2 instructions (two record values, two direction pairs or two components per
// instruction); FP64 takes the same steps one value at a time.
#pragma once

#include "nfe_fused2d.cuh"

namespace nfe {

template <int N, typename T, int TX, int TY>
struct Fused3DShape {
    static constexpr int AX = TX + 4, AY = TY + 4, APLANE = AX * AY;
    static constexpr int BX = TX + 2, BY = TY + 2, BPLANE = BX * BY;
    static constexpr int ASLOTS = 4, BSLOTS = 3;
    using RA = SRec<T, N>;               // evolved C (N-1), E_B
    using RB = SRec<T, 2 * N + 2>;       // evolved C (N-1), vx, vy, vz, S (N-1), |v|^2
    static constexpr int A_SLOT = RA::NVP * APLANE;
    static constexpr int B_SLOT = RB::NVP * BPLANE;
    static constexpr size_t BYTES = sizeof(T) * size_t(ASLOTS * A_SLOT + BSLOTS * B_SLOT);
    static constexpr int NHALO = BPLANE - TX * TY;
};

__device__ __forceinline__ int slotA(int z) { return (z + 8) & 3; }   // z >= -2
__device__ __forceinline__ int slotB(int z) { return (z + 9) % 3; }   // z >= -1

// Asynchronous global -> shared copies of one 4- or 8-byte value (cp.async, L1-allocating).
template <typename T>
__device__ __forceinline__ void cp_async_value(T *dst_smem, const T *src) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte values");
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst_smem));
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ----------------------------------------------------------------------------
// Stencil (Eqs. 35-36) from three A-planes (below, centre, above) at in-plane index ia.
// Out: the N volume fractions, their Laplacian and gradient (the implicit component's are
// minus the sums of the others), and grad E_B.  A neighbour beyond a wall contributes no
// difference (psi there := psi(x), Sec. III C).  With D3Q19 weights w_axis = 2 w_diag, every
// sum is accumulated in units of w_diag = 1/36: lap = 6 w_diag sum' = sum' / 6 and
// grad = 3 w_diag sum' = sum' / 12, where sum' counts axis neighbours twice.
// ----------------------------------------------------------------------------
template <int N, int AX, bool CHECK>
__device__ __forceinline__ void stencil3d_packed(const float *pm, const float *p0, const float *pp, int count, int ia,
                                                 unsigned wall, float (&c)[N], float (&lap)[N], float (&g)[N][3],
                                                 float (&gE)[3]) {
    using RA = SRec<float, N>;
    constexpr int NPU = (N + 1) / 2;     // value pairs holding the N used record values
    float r0[RA::NVP];
    srec_load<float, N>(p0, count, ia, r0);
    float2 L[NPU], GX[NPU], GY[NPU], GZ[NPU];
#pragma unroll
    for (int p = 0; p < NPU; ++p) L[p] = GX[p] = GY[p] = GZ[p] = make_float2(0.0f, 0.0f);
    const float2 two = dup2(2.0f), mtwo = dup2(-2.0f);
    sfor<1, 19, 1>([&](auto kc_) {
        constexpr int k = decltype(kc_)::value;
        constexpr int ex = LD3Q19::ex(k), ey = LD3Q19::ey(k), ez = LD3Q19::ez(k);
        constexpr bool axis = k < 7;
        if (CHECK && ((wall >> k) & 1u)) return;
        const float *pl = ez > 0 ? pp : (ez < 0 ? pm : p0);
        float r[RA::NVP];
        srec_load<float, N>(pl, count, ia + ex + AX * ey, r);
#pragma unroll
        for (int p = 0; p < NPU; ++p) {
            const float2 d = sub2(make_float2(r[2 * p], r[2 * p + 1]), make_float2(r0[2 * p], r0[2 * p + 1]));
            if constexpr (axis) {
                L[p] = fma2(two, d, L[p]);
                if constexpr (ex != 0) GX[p] = fma2(ex > 0 ? two : mtwo, d, GX[p]);
                if constexpr (ey != 0) GY[p] = fma2(ey > 0 ? two : mtwo, d, GY[p]);
                if constexpr (ez != 0) GZ[p] = fma2(ez > 0 ? two : mtwo, d, GZ[p]);
            } else {
                L[p] = add2(L[p], d);
                if constexpr (ex != 0) GX[p] = ex > 0 ? add2(GX[p], d) : sub2(GX[p], d);
                if constexpr (ey != 0) GY[p] = ey > 0 ? add2(GY[p], d) : sub2(GY[p], d);
                if constexpr (ez != 0) GZ[p] = ez > 0 ? add2(GZ[p], d) : sub2(GZ[p], d);
            }
        }
    });
    const float2 sixth = dup2(1.0f / 6.0f), twelfth = dup2(1.0f / 12.0f);
    float Lv[2 * NPU], Xv[2 * NPU], Yv[2 * NPU], Zv[2 * NPU];
#pragma unroll
    for (int p = 0; p < NPU; ++p) {
        const float2 l = mul2(sixth, L[p]), x = mul2(twelfth, GX[p]), y = mul2(twelfth, GY[p]), z = mul2(twelfth, GZ[p]);
        Lv[2 * p] = l.x; Lv[2 * p + 1] = l.y;
        Xv[2 * p] = x.x; Xv[2 * p + 1] = x.y;
        Yv[2 * p] = y.x; Yv[2 * p + 1] = y.y;
        Zv[2 * p] = z.x; Zv[2 * p + 1] = z.y;
    }
    float sl = 0.0f, sx = 0.0f, sy = 0.0f, sz = 0.0f, rest = 0.0f;
#pragma unroll
    for (int a = 0; a < N - 1; ++a) {
        c[a] = r0[a];
        rest += r0[a];
        lap[a] = Lv[a]; g[a][0] = Xv[a]; g[a][1] = Yv[a]; g[a][2] = Zv[a];
        sl += Lv[a]; sx += Xv[a]; sy += Yv[a]; sz += Zv[a];
    }
    c[N - 1] = 1.0f - rest;
    lap[N - 1] = -sl; g[N - 1][0] = -sx; g[N - 1][1] = -sy; g[N - 1][2] = -sz;
    gE[0] = Xv[N - 1]; gE[1] = Yv[N - 1]; gE[2] = Zv[N - 1];
}

template <int N, typename T, int AX, bool CHECK>
__device__ __forceinline__ void stencil3d(const T *pm, const T *p0, const T *pp, int count, int ia, unsigned wall,
                                          T (&c)[N], T (&lap)[N], T (&g)[N][3], T (&gE)[3]) {
    if constexpr (sizeof(T) == 4) {
        stencil3d_packed<N, AX, CHECK>(pm, p0, pp, count, ia, wall, c, lap, g, gE);
        return;
    }
    using RA = SRec<T, N>;
    T r0[RA::NVP];
    srec_load<T, N>(p0, count, ia, r0);
    T acc[N][4];          // lap, gx, gy, gz sums in units of w_diag (value N-1 = bulk energy: gradient only)
#pragma unroll
    for (int a = 0; a < N; ++a) acc[a][0] = acc[a][1] = acc[a][2] = acc[a][3] = T(0);
    sfor<1, 19, 1>([&](auto kc_) {
        constexpr int k = decltype(kc_)::value;
        constexpr int ex = LD3Q19::ex(k), ey = LD3Q19::ey(k), ez = LD3Q19::ez(k);
        constexpr bool axis = k < 7;
        if (CHECK && ((wall >> k) & 1u)) return;     // psi beyond a wall := psi(x)
        const T *pl = ez > 0 ? pp : (ez < 0 ? pm : p0);
        T r[RA::NVP];
        srec_load<T, N>(pl, count, ia + ex + AX * ey, r);
        const T wk = axis ? T(2) : T(1);
#pragma unroll
        for (int a = 0; a < N; ++a) {
            const T d = r[a] - r0[a];
            if (a < N - 1) acc[a][0] += wk * d;
            if constexpr (ex != 0) acc[a][1] += (ex > 0 ? wk : -wk) * d;
            if constexpr (ey != 0) acc[a][2] += (ey > 0 ? wk : -wk) * d;
            if constexpr (ez != 0) acc[a][3] += (ez > 0 ? wk : -wk) * d;
        }
    });
    T sl = T(0), sx = T(0), sy = T(0), sz = T(0), rest = T(0);
    const T sixth = T(1) / T(6), twelfth = T(1) / T(12);
#pragma unroll
    for (int a = 0; a < N - 1; ++a) {
        c[a] = r0[a];
        rest += r0[a];
        lap[a] = sixth * acc[a][0];
        g[a][0] = twelfth * acc[a][1]; g[a][1] = twelfth * acc[a][2]; g[a][2] = twelfth * acc[a][3];
        sl += lap[a]; sx += g[a][0]; sy += g[a][1]; sz += g[a][2];
    }
    c[N - 1] = T(1) - rest;
    lap[N - 1] = -sl; g[N - 1][0] = -sx; g[N - 1][1] = -sy; g[N - 1][2] = -sz;
    gE[0] = twelfth * acc[N - 1][1]; gE[1] = twelfth * acc[N - 1][2]; gE[2] = twelfth * acc[N - 1][3];
}

// Sums and differences of the direction pairs (k, k+1), k odd: sp[j] = f_k + f_k+1 and
// dm[j] = f_k - f_k+1 for pair j = (k - 1) / 2.  The moments and the TRT collision use only these.
// In FP32 the pairs are formed two at a time in the grouping the collision uses ((0, 1), (3, 4),
// (5, 6), (7, 8), and 2 alone), so that its packed operands need no regrouping.
template <typename T>
__device__ __forceinline__ void pair_sums(const T (&f)[19], T (&sp)[9], T (&dm)[9]) {
    if constexpr (sizeof(T) == 4) {
        auto two = [&](int j0, int j1) {
            const float2 a = make_float2(f[2 * j0 + 1], f[2 * j1 + 1]), b = make_float2(f[2 * j0 + 2], f[2 * j1 + 2]);
            const float2 s2 = add2(a, b), d2 = sub2(a, b);
            sp[j0] = s2.x; sp[j1] = s2.y; dm[j0] = d2.x; dm[j1] = d2.y;
        };
        two(0, 1);
        sp[2] = f[5] + f[6];
        dm[2] = f[5] - f[6];
        two(3, 4);
        two(5, 6);
        two(7, 8);
    } else {
#pragma unroll
        for (int j = 0; j < 9; ++j) { sp[j] = f[2 * j + 1] + f[2 * j + 2]; dm[j] = f[2 * j + 1] - f[2 * j + 2]; }
    }
}

// Force (Eq. 34, or Eq. 31 with cf.nonconservative), body forces, flux potential (Eq. 12)
// and moments (Eqs. 37-38) at one site.  f holds f_1..f_18; sp / dm are returned for the collision.
template <int N, typename T, int Q4>
__device__ __forceinline__ void site_physics3d(const Coef<T> &cf, const T (&c)[N], const T (&lap)[N],
                                               const T (&g)[N][3], const T (&gE)[3], const T (&f)[19],
                                               T (&S)[N - 1], T (&F)[3], T (&v)[3], T &P, T (&sp)[9], T (&dm)[9]) {
    if (!cf.nonconservative) {
        F[0] = gE[0]; F[1] = gE[1]; F[2] = gE[2];
#pragma unroll
        for (int a = 0; a < N; ++a) {
            T h = T(0);
#pragma unroll
            for (int b = 0; b < N; ++b) if (b != a) h += cf.kappa[a][b] * lap[b];
            F[0] += h * g[a][0]; F[1] += h * g[a][1]; F[2] += h * g[a][2];
        }
    } else {
        F[0] = F[1] = F[2] = T(0);
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
            F[0] += mu * g[a][0]; F[1] += mu * g[a][1]; F[2] += mu * g[a][2];
        }
    }
    F[0] += cf.fb[0]; F[1] += cf.fb[1]; F[2] += cf.fb[2];
    if (cf.has_fc) {
        // body force on one component, F += C_c F_c
        T cc = T(0);
#pragma unroll
        for (int a = 0; a < N; ++a) cc += cf.fcsel[a] * c[a];
        F[0] += cc * cf.fc[0]; F[1] += cc * cf.fc[1]; F[2] += cc * cf.fc[2];
    }
    T q[N - 1];
    flux_poly<N, T, Q4>(c, cf, q);
#pragma unroll
    for (int e = 0; e < N - 1; ++e) S[e] = c[e] * q[e] + cf.d34 * lap[e];
    flux_rest<N, T, Q4>(c, cf, S);     // the no-phi ablation's remainder (Q4_NOPHI only)
    // moments from the pair sums: pairs (1,2) (3,4) (5,6) are the axes, then xy (+,+) (+,-),
    // xz (+,+) (+,-), yz (+,+) (+,-), each pair's first direction listed
    pair_sums<T>(f, sp, dm);
    const T sumf = ((sp[0] + sp[1]) + (sp[2] + sp[3])) + ((sp[4] + sp[5]) + (sp[6] + sp[7])) + sp[8];
    const T jx = (dm[0] + (dm[3] + dm[4])) + (dm[5] + dm[6]);
    const T jy = (dm[1] + (dm[3] - dm[4])) + (dm[7] + dm[8]);
    const T jz = (dm[2] + (dm[5] - dm[6])) + (dm[7] - dm[8]);
    v[0] = jx + T(0.5) * F[0];
    v[1] = jy + T(0.5) * F[1];
    v[2] = jz + T(0.5) * F[2];
    // P = c_s^2 / (1 - w_0) [sum_{k != 0} f_k + s_0(v)], s_0 = -w_0 |v|^2 / (2 c_s^2)
    P = (sumf - T(0.5) * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2])) * T(0.5);
}

// TRT collision with forcing (Eqs. 23-30) of one site, regrouped so that per-site factors are
// formed once: for a pair (k, kbar), with s = f_k + f_kbar and d = f_k - f_kbar,
//   sym  = w_k [X + e.v (Y e.v + Z e.F)] - (op / 2) s
//   anti = w_k (U e.v + V e.F) - (om / 2) d
// where X = op (3P - 1.5 v.v) - 3 ap v.F, Y = 4.5 op, Z = 9 ap, U = 3 om, V = 3 am
// (ap = 1 - op / 2, am = 1 - om / 2).  Post-collision values replace f.
template <int N, typename T>
__device__ __forceinline__ void collide3d(const Coef<T> &cf, const T (&c)[N], const T (&v)[3], const T (&F)[3], T P,
                                          const T (&sp)[9], const T (&dm)[9], T (&f)[19]) {
    T op, om;
    relaxation<N, T>(cf, c, op, om);
    const T ap = T(1) - T(0.5) * op, am = T(1) - T(0.5) * om;
    const T vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const T vF = v[0] * F[0] + v[1] * F[1] + v[2] * F[2];
    const T X = op * (T(3) * P - T(1.5) * vv) - T(3) * ap * vF, Y = T(4.5) * op, Z = T(9) * ap, U = T(3) * om,
            V = T(3) * am;
    const T hop = T(0.5) * op, hom = T(0.5) * om;
    if constexpr (sizeof(T) == 4) {
        // two pairs of one weight class per instruction: (1,2)+(3,4), then (5,6) alone, then
        // the six diagonal pairs two by two; e.v and e.F of the first direction of each pair
        // formed two at a time (a + b and a - b as one packed FMA, exact)
        const float2 mhop = dup2(-hop), mhom = dup2(-hom);
        const float2 pm = make_float2(1.0f, -1.0f);
        const float2 eu2[5] = {make_float2(v[0], v[1]), make_float2(v[2], 0.0f), fma2(dup2(v[1]), pm, dup2(v[0])),
                               fma2(dup2(v[2]), pm, dup2(v[0])), fma2(dup2(v[2]), pm, dup2(v[1]))};
        const float2 eF2[5] = {make_float2(F[0], F[1]), make_float2(F[2], 0.0f), fma2(dup2(F[1]), pm, dup2(F[0])),
                               fma2(dup2(F[2]), pm, dup2(F[0])), fma2(dup2(F[2]), pm, dup2(F[1]))};
        auto two_pairs = [&](float wk, int j0, int j1, int q) {
            const float2 e_u = eu2[q], e_F = eF2[q];
            const float2 s = make_float2(sp[j0], sp[j1]), d = make_float2(dm[j0], dm[j1]);
            const float2 sym = fma2(mhop, s, fma2(e_u, fma2(dup2(wk * Y), e_u, mul2(dup2(wk * Z), e_F)), dup2(wk * X)));
            const float2 anti = fma2(mhom, d, fma2(dup2(wk * U), e_u, mul2(dup2(wk * V), e_F)));
            const float2 fk = make_float2(f[2 * j0 + 1], f[2 * j1 + 1]), fkb = make_float2(f[2 * j0 + 2], f[2 * j1 + 2]);
            const float2 pk = add2(fk, add2(sym, anti)), pkb = add2(fkb, sub2(sym, anti));
            f[2 * j0 + 1] = pk.x; f[2 * j1 + 1] = pk.y; f[2 * j0 + 2] = pkb.x; f[2 * j1 + 2] = pkb.y;
        };
        const float wa = float(LD3Q19::w(1)), wd = float(LD3Q19::w(7));
        two_pairs(wa, 0, 1, 0);
        {
            const float eu = v[2], eF = F[2];
            const float sym = (wa * X + eu * ((wa * Y) * eu + (wa * Z) * eF)) - hop * sp[2];
            const float anti = ((wa * U) * eu + (wa * V) * eF) - hom * dm[2];
            f[5] = f[5] + (sym + anti);
            f[6] = f[6] + (sym - anti);
        }
        two_pairs(wd, 3, 4, 2);
        two_pairs(wd, 5, 6, 3);
        two_pairs(wd, 7, 8, 4);
    } else {
        // e.v and e.F of the first direction of every pair
        const T eu[9] = {v[0], v[1], v[2], v[0] + v[1], v[0] - v[1], v[0] + v[2], v[0] - v[2], v[1] + v[2], v[1] - v[2]};
        const T eF[9] = {F[0], F[1], F[2], F[0] + F[1], F[0] - F[1], F[0] + F[2], F[0] - F[2], F[1] + F[2], F[1] - F[2]};
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const T wk = j < 3 ? T(LD3Q19::w(1)) : T(LD3Q19::w(7));
            const T sym = (wk * X + eu[j] * ((wk * Y) * eu[j] + (wk * Z) * eF[j])) - hop * sp[j];
            const T anti = ((wk * U) * eu[j] + (wk * V) * eF[j]) - hom * dm[j];
            f[2 * j + 1] = f[2 * j + 1] + (sym + anti);
            f[2 * j + 2] = f[2 * j + 2] + (sym - anti);
        }
    }
}

// |v|^2 with an explicit operation order, so that every kernel that forms it (the fused step's
// record, the split form's gather staging) gets the same bits.
template <typename T>
__device__ __forceinline__ T vsq3(T a, T b, T c) {
    if constexpr (sizeof(T) == 4) return __fmaf_rn(c, c, __fmaf_rn(b, b, __fmul_rn(a, a)));
    else return __fma_rn(c, c, __fma_rn(b, b, __dmul_rn(a, a)));
}

// Directions with e_kx > 0 (the links of a site of column nx - 1 into the outflow's ghost column).
__host__ __device__ constexpr unsigned d3q19_xplus_mask() {
    unsigned m = 0u;
    for (int k = 1; k < 19; ++k)
        if (LD3Q19::ex(k) > 0) m |= 1u << k;
    return m;
}

// Push-streaming of the post-collision populations of one own site s0 (in-plane wrapped
// coordinates sx, sy, plane zw) with halfway bounce-back (Eqs. 44-45) where wall0 has bit k set.
// The periodic wrap is folded into six per-site neighbour offsets, so every site of a warp runs
// the same store sequence; only sites next to a wall take the bounce-back form.
template <typename T, typename SF>
__device__ __forceinline__ void push_store3d(const Coef<T> &cf, SF *__restrict__ fout, int n, int nx, int ny, int nz,
                                             int sx, int sy, int zw, int s0, unsigned wall0, const T (&f)[19],
                                             bool checked = false, unsigned drop = 0u) {
    const int nxy = nx * ny;
    const int dxp = sx == nx - 1 ? 1 - nx : 1, dxm = sx == 0 ? nx - 1 : -1;
    const int dyp = sy == ny - 1 ? nx - nxy : nx, dym = sy == 0 ? nxy - nx : -nx;
    const int dzp = zw == nz - 1 ? nxy - n : nxy, dzm = zw == 0 ? n - nxy : -nxy;
    auto target = [&](auto kc_) {
        constexpr int k = decltype(kc_)::value;
        constexpr int ex = LD3Q19::ex(k), ey = LD3Q19::ey(k), ez = LD3Q19::ez(k);
        int t = s0;
        if constexpr (ex != 0) t += ex > 0 ? dxp : dxm;
        if constexpr (ey != 0) t += ey > 0 ? dyp : dym;
        if constexpr (ez != 0) t += ez > 0 ? dzp : dzm;
        return t;
    };
    // checked: the bounce-back form whatever wall0 (a warp-wide choice; same stores where wall0 = 0)
    if (wall0 == 0u && !checked) {
        sfor<1, 19, 1>([&](auto kc_) {
            constexpr int k = decltype(kc_)::value;
            FStore<SF, T>::store(fout + (k - 1) * n + target(kc_), f[k], LD3Q19::w(k), cf.fscale);
        });
    } else {
        sfor<1, 19, 1>([&](auto kc_) {
            constexpr int k = decltype(kc_)::value;
            constexpr int kb = opp(k);
            // halfway bounce-back: f_kbar(x, t+1) = post_k(x); a dropped link (into the outflow's
            // ghost column) stores nothing
            if ((wall0 >> k) & 1u) FStore<SF, T>::store(fout + (kb - 1) * n + s0, f[k], LD3Q19::w(kb), cf.fscale);
            else if (!((drop >> k) & 1u)) FStore<SF, T>::store(fout + (k - 1) * n + target(kc_), f[k], LD3Q19::w(k), cf.fscale);
        });
    }
}

// Shared-memory / scratch record of NV values over `count` sites: full 16-byte chunks in separate
// planes, then, for the values left over, an 8-byte plane (two FP32 values) and a plane of single
// values (one FP32 or FP64 value).  Every plane keeps consecutive sites consecutive.
template <typename T, int NV>
struct TRec {
    static constexpr int PER = 16 / sizeof(T);
    static constexpr int NC = NV / PER;            // full chunks
    static constexpr int TAIL = NV - NC * PER;     // 0..3 (FP32), 0..1 (FP64)
    static constexpr int TAIL2 = (sizeof(T) == 4 && TAIL >= 2) ? 2 : 0;   // values in the 8-byte plane
    static constexpr int TAIL1 = TAIL - TAIL2;                            // values in the single plane
    static constexpr int NVP = NV;
    // offsets (in values) of the planes for `count` sites
    __host__ __device__ static constexpr size_t chunk_at(int c, size_t count) { return size_t(c) * count * PER; }
    __host__ __device__ static constexpr size_t tail2_at(size_t count) { return size_t(NC) * count * PER; }
    __host__ __device__ static constexpr size_t tail1_at(size_t count) { return size_t(NC) * count * PER + TAIL2 * count; }
};

template <typename T, int NV, int NOUT>
__device__ __forceinline__ void trec_load(const T *base, int count, int i, T (&out)[NOUT]) {
    using R = TRec<T, NV>;
    using V = typename Vec16<T>::type;
#pragma unroll
    for (int c = 0; c < R::NC; ++c) {
        const V v = reinterpret_cast<const V *>(base + R::chunk_at(c, count))[i];
        if constexpr (sizeof(T) == 4) {
            out[4 * c + 0] = v.x; out[4 * c + 1] = v.y; out[4 * c + 2] = v.z; out[4 * c + 3] = v.w;
        } else {
            out[2 * c + 0] = v.x; out[2 * c + 1] = v.y;
        }
    }
    if constexpr (R::TAIL2 == 2) {
        const float2 v = reinterpret_cast<const float2 *>(base + R::tail2_at(count))[i];
        out[R::NC * R::PER] = v.x; out[R::NC * R::PER + 1] = v.y;
    }
    if constexpr (R::TAIL1 == 1) out[R::NC * R::PER + R::TAIL2] = (base + R::tail1_at(count))[i];
}

template <typename T, int NV, int NIN>
__device__ __forceinline__ void trec_store(T *base, size_t count, size_t i, const T (&in)[NIN]) {
    using R = TRec<T, NV>;
    using V = typename Vec16<T>::type;
#pragma unroll
    for (int c = 0; c < R::NC; ++c) {
        V w;
        if constexpr (sizeof(T) == 4) { w.x = in[4 * c]; w.y = in[4 * c + 1]; w.z = in[4 * c + 2]; w.w = in[4 * c + 3]; }
        else { w.x = in[2 * c]; w.y = in[2 * c + 1]; }
        reinterpret_cast<V *>(base + R::chunk_at(c, count))[i] = w;
    }
    if constexpr (R::TAIL2 == 2)
        reinterpret_cast<float2 *>(base + R::tail2_at(count))[i] = make_float2(in[R::NC * R::PER], in[R::NC * R::PER + 1]);
    if constexpr (R::TAIL1 == 1) (base + R::tail1_at(count))[i] = in[R::NC * R::PER + R::TAIL2];
}

// The B record (C, v, S, |v|^2) of one site, loaded into NV = 2N + 2 values: from SRec planes
// holding all of them (fused step, SLIM false), or from TRec planes without |v|^2 (split step,
// SLIM true: the gather record in HBM and shared memory is one value shorter and |v|^2 is formed
// after the load, with the same operations as where the fused step forms it).
template <typename T, int NV, bool SLIM>
struct BRec {
    static constexpr int NVP = SLIM ? NV : SRec<T, NV>::NVP;
    __device__ __forceinline__ static void load(const T *base, int count, int i, T (&out)[NVP]) {
        if constexpr (SLIM) {
            trec_load<T, NV - 1>(base, count, i, out);
            constexpr int N = (NV - 2) / 2;
            out[NV - 1] = vsq3<T>(out[N - 1], out[N], out[N + 1]);
        } else {
            srec_load<T, NV>(base, count, i, out);
        }
    }
};

// Order in which the Cahn-Hilliard gather visits its 18 sources y = x - e_k: the directions k
// sorted by the source offset -e_k in (z, y, x) order.  A gather of two sites stacked in y visits
// the union of their sources in the same order, so each site sums its terms in this order too.
constexpr int kGatherOrder[18] = {15, 11, 5, 14, 18, 7, 3, 10, 1, 2, 9, 4, 8, 17, 13, 6, 12, 16};

// The D3Q19 direction k with e_k = (x, y, z): 1..18, 0 for the rest velocity, -1 if none.
__host__ __device__ constexpr int d3q19_dir(int x, int y, int z) {
    for (int k = 0; k < 19; ++k)
        if (LD3Q19::ex(k) == x && LD3Q19::ey(k) == y && LD3Q19::ez(k) == z) return k;
    return -1;
}

// FMA and product with the rounding fixed: a gather's terms are summed by different code in the
// one-site and the stacked forms, and an expression left to the compiler may be contracted
// differently in each; these keep every form on the same bits.
template <typename T>
__device__ __forceinline__ T fma_x(T a, T b, T c) {
    if constexpr (sizeof(T) == 4) return __fmaf_rn(a, b, c);
    else return __fma_rn(a, b, c);
}
template <typename T>
__device__ __forceinline__ T mul_x(T a, T b) {
    if constexpr (sizeof(T) == 4) return __fmul_rn(a, b);
    else return __dmul_rn(a, b);
}

// s_k(v) = w_k (3 eu + 4.5 eu^2 - 1.5 |v|^2) = eu (3 w_k + 4.5 w_k eu) - 1.5 w_k |v|^2, eu = e_k . v
// (the velocity part of g^eq_k, Eq. 40), with a fixed rounding sequence.
template <typename T, int k>
__device__ __forceinline__ T s_of(T eu, T vsq) {
    return fma_x(eu, fma_x(T(4.5 * LD3Q19::w(k)), eu, T(3.0 * LD3Q19::w(k))), mul_x(T(-1.5 * LD3Q19::w(k)), vsq));
}

// One source term of the Cahn-Hilliard gather: record r of the source y = x - e_k adds
// C_i(y) s_k(v(y)) to acc and w_k (S_i(y) - S_i(x)) to lapS (r0: the record of x).
template <int N, typename T, int k, int NVP>
__device__ __forceinline__ void gather_term(const T (&r)[NVP], const T (&r0)[NVP], T (&acc)[N - 1], T (&lapS)[N - 1]) {
    constexpr int E = N - 1;
    constexpr int ex = LD3Q19::ex(k), ey = LD3Q19::ey(k), ez = LD3Q19::ez(k);
    const T wk = T(LD3Q19::w(k));
    // e_k . v(y) with the constant components folded (each is 0 or +-1)
    T eu = T(0);
    if constexpr (ex != 0) eu = ex > 0 ? r[N - 1] : -r[N - 1];
    if constexpr (ey != 0) eu = ey > 0 ? eu + r[N] : eu - r[N];
    if constexpr (ez != 0) eu = ez > 0 ? eu + r[N + 1] : eu - r[N + 1];
    const T sk = s_of<T, k>(eu, r[2 * N + 1]);
    if constexpr (sizeof(T) == 4) {
#pragma unroll
        for (int e = 0; e + 1 < E; e += 2) {
            const float2 cy = make_float2(r[e], r[e + 1]);
            const float2 ds = sub2(make_float2(r[N + 2 + e], r[N + 3 + e]), make_float2(r0[N + 2 + e], r0[N + 3 + e]));
            const float2 a = fma2(cy, dup2(sk), make_float2(acc[e], acc[e + 1]));
            const float2 l = fma2(dup2(float(LD3Q19::w(k))), ds, make_float2(lapS[e], lapS[e + 1]));
            acc[e] = a.x; acc[e + 1] = a.y; lapS[e] = l.x; lapS[e + 1] = l.y;
        }
        if constexpr (E % 2 == 1) {
            acc[E - 1] = fma_x(r[E - 1], sk, acc[E - 1]);
            lapS[E - 1] = fma_x(wk, r[N + 1 + E] - r0[N + 1 + E], lapS[E - 1]);
        }
    } else {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            acc[e] = fma_x(r[e], sk, acc[e]);
            lapS[e] = fma_x(wk, r[N + 2 + e] - r0[N + 2 + e], lapS[e]);
        }
    }
}

// The bounce-back term of direction k (source beyond a wall): the link carries g^eq_kbar(x),
// C_i(x) s_kbar(v(x)), and no S difference.
template <int N, typename T, int k, int NVP>
__device__ __forceinline__ void bounce_term(const T (&r0)[NVP], T (&acc)[N - 1]) {
    constexpr int ex = LD3Q19::ex(k), ey = LD3Q19::ey(k), ez = LD3Q19::ez(k);
    // e_kbar . v(x) = -e_k . v(x), the constant components folded
    T eu = T(0);
    if constexpr (ex != 0) eu = ex > 0 ? -r0[N - 1] : r0[N - 1];
    if constexpr (ey != 0) eu = ey > 0 ? eu - r0[N] : eu + r0[N];
    if constexpr (ez != 0) eu = ez > 0 ? eu - r0[N + 1] : eu + r0[N + 1];
    const T sk = s_of<T, k>(eu, r0[2 * N + 1]);
#pragma unroll
    for (int e = 0; e < N - 1; ++e) acc[e] = fma_x(r0[e], sk, acc[e]);
}

// Start of a gather: the rest population's increment C_i(x) s_0(v(x)).
template <int N, typename T, int NVP>
__device__ __forceinline__ void gather_init(const T (&r0)[NVP], T (&acc)[N - 1], T (&lapS)[N - 1]) {
    const T s0 = mul_x(T(-0.5), r0[2 * N + 1]);      // -1.5 w_0 |v|^2, w_0 = 1/3
#pragma unroll
    for (int e = 0; e < N - 1; ++e) { acc[e] = mul_x(r0[e], s0); lapS[e] = T(0); }
}

// End of a gather: C(x) + increments, the S Laplacian as link differences (mass-exact).
template <int N, typename T, int NVP>
__device__ __forceinline__ void gather_final(const T (&r0)[NVP], const T (&acc)[N - 1], const T (&lapS)[N - 1], T m,
                                             T (&out)[N - 1]) {
#pragma unroll
    for (int e = 0; e < N - 1; ++e) out[e] = r0[e] + fma_x(-m, lapS[e], acc[e]);
}

// Cahn-Hilliard update (Eqs. 39-41, tau_g = 1) of one site from the (C, v, S, |v|^2) records of
// three planes (below, centre, above) at in-plane index ib (row pitch BX):
// C_i(x, t+1) = C_i(x) + sum_k C_i(y) s_k(v(y)) + m sum_{k != 0} w_k (S_i(x) - S_i(y)), y = x - e_k,
// the increments gathered before C(x) is added and the S Laplacian as link differences, so
// that every link's two contributions cancel exactly.  A source beyond a wall bounces back
// (wall0 bit kbar set for the source x - e_k = x + e_kbar).
template <int N, typename T, int BX, bool CHECK, bool SLIM = false>
__device__ __forceinline__ void gather3d(const T *bm, const T *b0, const T *bp, int bplane, int ib, unsigned wall0,
                                         T m, T (&out)[N - 1]) {
    using RB = BRec<T, 2 * N + 2, SLIM>;
    T r0[RB::NVP];
    RB::load(b0, bplane, ib, r0);
    T acc[N - 1], lapS[N - 1];
    gather_init<N, T>(r0, acc, lapS);
    sfor<0, 18, 1>([&](auto jc_) {
        constexpr int k = kGatherOrder[decltype(jc_)::value];
        constexpr int kb = opp(k);
        if (CHECK && ((wall0 >> kb) & 1u)) {
            bounce_term<N, T, k>(r0, acc);
        } else {
            const T *pl = LD3Q19::ez(kb) > 0 ? bp : (LD3Q19::ez(kb) < 0 ? bm : b0);
            T r[RB::NVP];
            RB::load(pl, bplane, ib + LD3Q19::ex(kb) + BX * LD3Q19::ey(kb), r);
            gather_term<N, T, k>(r, r0, acc, lapS);
        }
    });
    gather_final<N, T>(r0, acc, lapS, m, out);
}

// Stored component populations (tau_g != 1, Sec. III B), one site x with global index s0 (in-plane
// wrapped coordinates sx, sy, plane z): g_{i,k}(x, t+1) = g*_{i,k}(x - e_k), g* = g + (g^eq - g) / tau_g,
// with g^eq_{i,k}(x - e_k) (Eq. 40 as read: C_i s_k(v) - w_k m S_i, and C_i (1 + s_0(v)) + (1 - w_0) m S_i
// for k = 0) from the source's record in shared memory and g from gin; a source beyond a wall gives
// g*_{i,kbar}(x) (Eqs. 44-45).  Writes all 19 populations of every evolved component to gout and
// returns C_i(x, t+1) = sum_k g_{i,k}(x, t+1) (Eq. 41).  Layout of g: plane (i 19 + k).
template <int N, typename T, int BX, bool CHECK, bool SLIM>
__device__ __forceinline__ void gather3d_taug(const T *bm, const T *b0, const T *bp, int bplane, int ib, unsigned wall0,
                                              T m, T omg, const T *__restrict__ gin, T *__restrict__ gout, int n,
                                              int nx, int ny, int nz, int sx, int sy, int z, int s0, T (&out)[N - 1]) {
    using RB = BRec<T, 2 * N + 2, SLIM>;
    constexpr int E = N - 1;
    const int nxy = nx * ny;
    // offsets to the sources x - e_k, periodic wrap folded in
    const int sxm = sx == 0 ? nx - 1 : -1, sxp = sx == nx - 1 ? 1 - nx : 1;
    const int sym = sy == 0 ? nxy - nx : -nx, syp = sy == ny - 1 ? nx - nxy : nx;
    const int szm = z == 0 ? n - nxy : -nxy, szp = z == nz - 1 ? nxy - n : nxy;
    T r0[RB::NVP];
    RB::load(b0, bplane, ib, r0);
#pragma unroll
    for (int e = 0; e < E; ++e) out[e] = T(0);
    sfor<0, 19, 1>([&](auto kc_) {
        constexpr int k = decltype(kc_)::value;
        constexpr int ex = LD3Q19::ex(k), ey = LD3Q19::ey(k), ez = LD3Q19::ez(k);
        const T wk = T(LD3Q19::w(k));
        if constexpr (k == 0) {
            const T s0k = wk * (-T(1.5) * r0[2 * N + 1]);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const T geq = r0[e] * (T(1) + s0k) + (T(1) - wk) * m * r0[N + 2 + e];
                const T gg = gin[size_t(e * 19) * n + s0];
                const T post = gg + omg * (geq - gg);
                gout[size_t(e * 19) * n + s0] = post;
                out[e] += post;
            }
        } else {
            constexpr int kb = opp(k);
            if (CHECK && ((wall0 >> kb) & 1u)) {
                // the source is beyond a wall: g_k(x, t+1) = g*_kbar(x)
                const T eu = T(LD3Q19::ex(kb)) * r0[N - 1] + T(LD3Q19::ey(kb)) * r0[N] + T(LD3Q19::ez(kb)) * r0[N + 1];
                const T skb = wk * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * r0[2 * N + 1]);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const T geq = r0[e] * skb - wk * m * r0[N + 2 + e];
                    const T gg = gin[size_t(e * 19 + kb) * n + s0];
                    const T post = gg + omg * (geq - gg);
                    gout[size_t(e * 19 + k) * n + s0] = post;
                    out[e] += post;
                }
            } else {
                const T *pl = ez < 0 ? bp : (ez > 0 ? bm : b0);      // the source is x - e_k
                T r[RB::NVP];
                RB::load(pl, bplane, ib - ex - BX * ey, r);
                const T eu = T(ex) * r[N - 1] + T(ey) * r[N] + T(ez) * r[N + 1];
                const T sk = wk * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * r[2 * N + 1]);
                int src = s0;
                if constexpr (ex != 0) src += ex > 0 ? sxm : sxp;
                if constexpr (ey != 0) src += ey > 0 ? sym : syp;
                if constexpr (ez != 0) src += ez > 0 ? szm : szp;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const T geq = r[e] * sk - wk * m * r[N + 2 + e];
                    const T gg = gin[size_t(e * 19 + k) * n + src];
                    const T post = gg + omg * (geq - gg);
                    gout[size_t(e * 19 + k) * n + s0] = post;
                    out[e] += post;
                }
            }
        }
    });
}

// Is the position (dx, dy, dz) relative to site 0 of a stack of K sites a source of one of them?
__host__ __device__ constexpr bool stack_source(int K, int dx, int dy, int dz) {
    for (int j = 0; j < K; ++j)
        if (d3q19_dir(-dx, j - dy, -dz) > 0) return true;
    return false;
}

// The same update for K sites stacked in y (site j at ib + j BX), sharing the loads of the records
// several of them need: 9 K + 10 record loads for the K sites instead of 19 K (28 for two sites,
// 37 for three, 46 for four).  The union of the sources is visited in (z, y, x) order, so each site
// still sums its terms in the order of kGatherOrder, as the one-site form does: all give the same
// bits.
template <int N, typename T, int BX, bool CHECK, bool SLIM, int K>
__device__ __forceinline__ void gather3d_stack(const T *bm, const T *b0, const T *bp, int bplane, int ib,
                                               const unsigned (&wall)[K], T m, T (&out)[K][N - 1]) {
    using RB = BRec<T, 2 * N + 2, SLIM>;
    T rs[K][RB::NVP];
#pragma unroll
    for (int j = 0; j < K; ++j) RB::load(b0, bplane, ib + j * BX, rs[j]);
    T acc[K][N - 1], lap[K][N - 1];
#pragma unroll
    for (int j = 0; j < K; ++j) gather_init<N, T>(rs[j], acc[j], lap[j]);
    // positions (dx, dy, dz) relative to site 0, dz then dy in -1..K then dx ascending
    constexpr int NYP = K + 2;
    sfor<0, 9 * NYP, 1>([&](auto pc_) {
        constexpr int pidx = decltype(pc_)::value;
        constexpr int dz = pidx / (3 * NYP) - 1, dy = (pidx / 3) % NYP - 1, dx = pidx % 3 - 1;
        // is this position a source of any of the K sites (a D3Q19 neighbour offset, not the site)?
        constexpr bool any = stack_source(K, dx, dy, dz);
        if constexpr (any) {
            // the records of the K sites themselves are already in registers
            constexpr int own = (dx == 0 && dz == 0 && dy >= 0 && dy < K) ? dy : -1;
            T r[RB::NVP];
            if constexpr (own >= 0) {
#pragma unroll
                for (int q = 0; q < RB::NVP; ++q) r[q] = rs[own][q];
            } else {
#pragma unroll
                for (int q = 0; q < RB::NVP; ++q) r[q] = T(0);
                // load unless every site that takes this source bounces back instead
                bool need = false;
                sfor<0, K, 1>([&](auto jc_) {
                    constexpr int j = decltype(jc_)::value;
                    constexpr int kj = d3q19_dir(-dx, j - dy, -dz);
                    if constexpr (kj > 0) need |= !(CHECK && ((wall[j] >> opp(kj)) & 1u));
                });
                if (need) {
                    const T *pl = dz > 0 ? bp : (dz < 0 ? bm : b0);
                    RB::load(pl, bplane, ib + dx + BX * dy, r);
                }
            }
            sfor<0, K, 1>([&](auto jc_) {
                constexpr int j = decltype(jc_)::value;
                constexpr int kj = d3q19_dir(-dx, j - dy, -dz);
                if constexpr (kj > 0) {
                    if (CHECK && ((wall[j] >> opp(kj)) & 1u)) bounce_term<N, T, kj>(rs[j], acc[j]);
                    else gather_term<N, T, kj>(r, rs[j], acc[j], lap[j]);
                }
            });
        }
    });
#pragma unroll
    for (int j = 0; j < K; ++j) gather_final<N, T>(rs[j], acc[j], lap[j], m, out[j]);
}

// Bit k set when x + e_k lies beyond a wall.
__device__ __forceinline__ unsigned wall_mask3(const Geom &g, int x, int y, int z) {
    unsigned m = 0;
    sfor<1, 19, 1>([&](auto kc_) {
        constexpr int k = decltype(kc_)::value;
        const int xx = x + LD3Q19::ex(k), yy = y + LD3Q19::ey(k), zz = z + LD3Q19::ez(k);
        if ((g.wx && (xx < 0 || xx >= g.nx)) || (g.wy && (yy < 0 || yy >= g.ny)) || (g.wz && (zz < 0 || zz >= g.nz)))
            m |= 1u << k;
    });
    return m;
}

// Per-thread state of one CTA of the fused D3Q19 step, and its phases.
template <int N, typename T, typename SF, int TX, int TY, int Q4>
struct Fused3DTile {
    using Sh = Fused3DShape<N, T, TX, TY>;
    using RA = typename Sh::RA;
    using RB = typename Sh::RB;
    static_assert(Sh::NHALO <= TX * TY, "one ring site per thread at most");
    static constexpr int NT = TX * TY;
    static constexpr int ITER = (Sh::APLANE + NT - 1) / NT;

    const Geom &g;
    const Coef<T> &cf;
    const SF *__restrict__ fin;
    SF *__restrict__ fout;
    const T *__restrict__ Cin;
    T *__restrict__ Cout;
    int *__restrict__ flag;
    T *sA, *sB;
    int nx, ny, nz, nxy, n, tid, x0, y0, z_lo, z_hi;
    bool edge;      // the tile plus its 2-ring crosses a domain edge (indices wrap or clamp)
    bool wallt;     // ... and that edge is a wall in x or y (stencils need wall tests)
    bool tiny;      // the domain is narrower than a tile plus ring: wrap with a full modulo
    // own site in the plane, and this thread's ring site
    int tx, ty, gx0, gy0, sx, sy, sxy, bx, by, hx, hy, hxy;
    bool own_xy, ring_xy_ok;
    int aoff[ITER];      // in-plane index (x + nx y) of this thread's A-sites, -1 past the plane

    __device__ __forceinline__ Fused3DTile(const Geom &g_, const Coef<T> &cf_, const SF *fin_, SF *fout_,
                                           const T *Cin_, T *Cout_, int *flag_, unsigned char *smem, int zchunk)
        : g(g_), cf(cf_), fin(fin_), fout(fout_), Cin(Cin_), Cout(Cout_), flag(flag_) {
        sA = reinterpret_cast<T *>(smem);
        sB = sA + Sh::ASLOTS * Sh::A_SLOT;
        nx = g.nx; ny = g.ny; nz = g.nz;
        nxy = nx * ny;
        n = int(g.n);
        tid = threadIdx.x;
        x0 = blockIdx.x * TX;
        y0 = blockIdx.y * TY;
        z_lo = blockIdx.z * zchunk;
        z_hi = min(z_lo + zchunk, nz);
        edge = (x0 - 2 < 0) || (x0 + TX + 2 > nx) || (y0 - 2 < 0) || (y0 + TY + 2 > ny);
        wallt = (g.wx && ((x0 - 2 < 0) || (x0 + TX + 2 > nx))) || (g.wy && ((y0 - 2 < 0) || (y0 + TY + 2 > ny)));
        tiny = nx < TX + 4 || ny < TY + 4;
        tx = tid % TX;
        ty = tid / TX;
        gx0 = x0 + tx;
        gy0 = y0 + ty;
        own_xy = gx0 < nx && gy0 < ny;
        sx = edge ? pwrap(gx0, nx, tiny) : gx0;
        sy = edge ? pwrap(gy0, ny, tiny) : gy0;
        sxy = sx + nx * sy;
        bx = 0;
        by = 0;
        const bool has_ring = tid < Sh::NHALO;
        if (tid < Sh::BX) { bx = tid; by = 0; }
        else if (tid < 2 * Sh::BX) { bx = tid - Sh::BX; by = Sh::BY - 1; }
        else { const int r = tid - 2 * Sh::BX; by = 1 + (r >> 1); bx = (r & 1) ? Sh::BX - 1 : 0; }
        hx = x0 + bx - 1;
        hy = y0 + by - 1;
        ring_xy_ok = has_ring && !(edge && ((g.wx && (hx < 0 || hx >= nx)) || (g.wy && (hy < 0 || hy >= ny))));
        hxy = edge ? pwrap(hx, nx, tiny) + nx * pwrap(hy, ny, tiny) : hx + nx * hy;
        // the A-sites this thread copies and completes in every plane (the same ones: the
        // completion reads only this thread's own copies, so it needs no barrier)
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int i = tid + it * NT;
            if (i < Sh::APLANE) {
                const int ly = i / Sh::AX, lx = i - ly * Sh::AX;
                int gx = x0 + lx - 2, gy = y0 + ly - 2;
                if (edge) {
                    gx = g.wx ? min(max(gx, 0), nx - 1) : pwrap(gx, nx, tiny);
                    gy = g.wy ? min(max(gy, 0), ny - 1) : pwrap(gy, ny, tiny);
                }
                aoff[it] = gx + nx * gy;
            } else {
                aoff[it] = -1;
            }
        }
    }

    // Periodic plane index of z in [z_lo - 2, z_hi + 2) without a division.
    __device__ __forceinline__ int zwrap(int z) const { return nz > 1 ? wrap(z, nz) : 0; }

    // copy_A: start the cp.async copies of the evolved C of A-plane za (tile + 2-ring) into its
    // slot and commit them as one group (an empty group beyond a z wall: never read).
    __device__ __forceinline__ void copy_A(int za) {
        if (!(g.wz && (za < 0 || za >= nz))) {
            const int zo = nxy * zwrap(za);
            T *base = sA + slotA(za) * Sh::A_SLOT;
#pragma unroll
            for (int it = 0; it < ITER; ++it) {
                const int i = tid + it * NT;
                if (aoff[it] >= 0) {
                    const int s = aoff[it] + zo;
#pragma unroll
                    for (int a = 0; a < N - 1; ++a)
                        cp_async_value<T>(base + (a / RA::PER) * Sh::APLANE * RA::PER + i * RA::PER + (a % RA::PER),
                                          Cin + size_t(a) * n + s);
                }
            }
        }
        cp_async_commit();
    }

    // finish_A: after this thread's copies of A-plane za have landed, E_B (Eq. 5) of its A-sites.
    __device__ __forceinline__ void finish_A(int za) {
        if (g.wz && (za < 0 || za >= nz)) return;      // beyond a wall: never read
        T *base = sA + slotA(za) * Sh::A_SLOT;
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int i = tid + it * NT;
            if (aoff[it] >= 0) {
                T rec[RA::NVP];
                srec_load<T, N>(base, Sh::APLANE, i, rec);
                T cc[N];
                T rest = T(0);
#pragma unroll
                for (int a = 0; a < N - 1; ++a) { cc[a] = rec[a]; rest += rec[a]; }
                cc[N - 1] = T(1) - rest;
                base[((N - 1) / RA::PER) * Sh::APLANE * RA::PER + i * RA::PER + ((N - 1) % RA::PER)] =
                    bulk_energy<N, T>(cc, cf);
            }
        }
    }

    // load_F: f of the own site and of the ring site of plane zb into registers (consumed by
    // fill_B one iteration later, so that HBM latency overlaps the gather of the plane below).
    __device__ __forceinline__ void load_F(int zb, T (&fo)[19], T (&fr)[19]) {
        fo[0] = fr[0] = T(0);
        if (g.wz && (zb < 0 || zb >= nz)) return;
        const int zw = zwrap(zb);
        const int s0 = sxy + nxy * zw;
        sfor<1, 19, 1>([&](auto kc_) { constexpr int k = decltype(kc_)::value; fo[k] = FStore<SF, T>::load(fin + (k - 1) * n + s0, LD3Q19::w(k), cf.finv); });
        if (ring_xy_ok) {
            const int s = hxy + nxy * zw;
            sfor<1, 19, 1>([&](auto kc_) { constexpr int k = decltype(kc_)::value; fr[k] = FStore<SF, T>::load(fin + (k - 1) * n + s, LD3Q19::w(k), cf.finv); });
        }
    }

    // B record of one site: C, v, S and |v|^2 (read 18 times by the gather)
    __device__ __forceinline__ void store_B(T *bbase, int ib, const T (&c)[N], const T (&v)[3], const T (&S)[N - 1]) {
        T rec[RB::NVP];
#pragma unroll
        for (int a = 0; a < N - 1; ++a) { rec[a] = c[a]; rec[N + 2 + a] = S[a]; }
        rec[N - 1] = v[0]; rec[N] = v[1]; rec[N + 1] = v[2];
        rec[2 * N + 1] = vsq3<T>(v[0], v[1], v[2]);
#pragma unroll
        for (int a = 2 * N + 2; a < RB::NVP; ++a) rec[a] = T(0);
        srec_store<T, 2 * N + 2>(bbase, Sh::BPLANE, ib, rec);
    }

    // fo is consumed: the collision leaves post-collision values in it
    __device__ __forceinline__ void fill_B(int zb, bool collide, T (&fo)[19], const T (&fr)[19]) {
        if (g.wz && (zb < 0 || zb >= nz)) return;      // sources beyond a wall bounce back
        const int zw = zwrap(zb);
        const T *pm = sA + slotA(zb - 1) * Sh::A_SLOT;
        const T *p0 = sA + slotA(zb) * Sh::A_SLOT;
        const T *pp = sA + slotA(zb + 1) * Sh::A_SLOT;
        T *bbase = sB + slotB(zb) * Sh::B_SLOT;
        const bool zcheck = g.wz && (zb == 0 || zb == nz - 1);
        const bool check = wallt || zcheck;
        // own site
        {
            const int s0 = sxy + nxy * zw;
            T (&f)[19] = fo;
            const unsigned wall0 = check ? wall_mask3(g, gx0, gy0, zb) : 0u;
            T c[N], lap[N], gr[N][3], gE[3];
            const int ia = (ty + 2) * Sh::AX + (tx + 2);
            if (check) stencil3d<N, T, Sh::AX, true>(pm, p0, pp, Sh::APLANE, ia, wall0, c, lap, gr, gE);
            else       stencil3d<N, T, Sh::AX, false>(pm, p0, pp, Sh::APLANE, ia, 0u, c, lap, gr, gE);
            T S[N - 1], F[3], v[3], P, sp[9], dm[9];
            site_physics3d<N, T, Q4>(cf, c, lap, gr, gE, f, S, F, v, P, sp, dm);
            store_B(bbase, (ty + 1) * Sh::BX + (tx + 1), c, v, S);
            if (collide && own_xy) {
                collide3d<N, T>(cf, c, v, F, P, sp, dm, f);
                push_store3d<T, SF>(cf, fout, n, nx, ny, nz, sx, sy, zw, s0, wall0, f);
            }
        }
        // ring site
        if (ring_xy_ok) {
            const unsigned wall = check ? wall_mask3(g, hx, hy, zb) : 0u;
            T c[N], lap[N], gr[N][3], gE[3];
            const int ia = (by + 1) * Sh::AX + (bx + 1);
            if (check) stencil3d<N, T, Sh::AX, true>(pm, p0, pp, Sh::APLANE, ia, wall, c, lap, gr, gE);
            else       stencil3d<N, T, Sh::AX, false>(pm, p0, pp, Sh::APLANE, ia, 0u, c, lap, gr, gE);
            T S[N - 1], F[3], v[3], P, sp[9], dm[9];
            site_physics3d<N, T, Q4>(cf, c, lap, gr, gE, fr, S, F, v, P, sp, dm);
            store_B(bbase, by * Sh::BX + bx, c, v, S);
        }
    }

    // Cahn-Hilliard update of the own site of plane zc from B-planes zc-1..zc+1
    template <bool CHECK>
    __device__ __forceinline__ void ch_impl(int zc, unsigned wall0) {
        T out[N - 1];
        gather3d<N, T, Sh::BX, CHECK>(sB + slotB(zc - 1) * Sh::B_SLOT, sB + slotB(zc) * Sh::B_SLOT,
                                      sB + slotB(zc + 1) * Sh::B_SLOT, Sh::BPLANE, (ty + 1) * Sh::BX + (tx + 1),
                                      wall0, cf.m, out);
        const int s0 = sxy + nxy * zc;
        bool bad = false;
#pragma unroll
        for (int e = 0; e < N - 1; ++e) {
            Cout[e * n + s0] = out[e];
            bad |= !isfinite(out[e]);
        }
        if (bad) atomicOr(flag, 1);
    }

    // the wall-free form carries no bounce-back code (no predicated second path); the form is
    // decided per site (not per tile), so a site runs the same code under every tile shape
    __device__ __forceinline__ void ch(int zc) {
        if (!own_xy) return;
        const unsigned wall0 = (wallt || (g.wz && (zc == 0 || zc == nz - 1))) ? wall_mask3(g, gx0, gy0, zc) : 0u;
        if (wall0) ch_impl<true>(zc, wall0);
        else ch_impl<false>(zc, 0u);
    }

    __device__ __forceinline__ void march() {
        T fo[19], fr[19];
        // warm-up: A-planes z_lo-2 .. z_lo+1 (all four slots), B-planes z_lo-1 and z_lo
#pragma unroll 1
        for (int za = z_lo - 2; za <= z_lo + 1; ++za) copy_A(za);
        load_F(z_lo - 1, fo, fr);
        cp_async_wait_all();
#pragma unroll 1
        for (int za = z_lo - 2; za <= z_lo + 1; ++za) finish_A(za);
        __syncthreads();
        fill_B(z_lo - 1, false, fo, fr);
        load_F(z_lo, fo, fr);
        fill_B(z_lo, true, fo, fr);
        __syncthreads();                      // A-plane z_lo - 2 is free
        copy_A(z_lo + 2);
        load_F(z_lo + 1, fo, fr);
#pragma unroll 1
        for (int zc = z_lo; zc < z_hi; ++zc) {
            cp_async_wait_all();
            finish_A(zc + 2);
            __syncthreads();
            fill_B(zc + 1, zc + 1 < z_hi, fo, fr);
            __syncthreads();
            if (zc + 1 < z_hi) {               // next plane's copies and loads fly while this plane is gathered
                copy_A(zc + 3);
                load_F(zc + 2, fo, fr);
            }
            ch(zc);
        }
    }
};

// Minimum resident CTAs per SM for the register allocator: as many as the shared
// memory admits, at most 512 threads per SM in FP32 (128 registers a thread).
template <int N, typename T, int TX, int TY>
struct Fused3DOcc {
    static constexpr int by_smem = int((227 * 1024) / (Fused3DShape<N, T, TX, TY>::BYTES + 1024));
    static constexpr int by_regs = sizeof(T) == 4 ? 512 / (TX * TY) : 256 / (TX * TY);
    static constexpr int value = by_smem < 1 ? 1 : (by_smem < by_regs ? by_smem : by_regs);
};

template <int N, typename T, typename SF, int TX, int TY, int Q4>
__global__ void __launch_bounds__(TX * TY, (Fused3DOcc<N, T, TX, TY>::value))
k_fused3d(Geom g, Coef<T> cf, const SF *__restrict__ fin, SF *__restrict__ fout,
          const T *__restrict__ Cin, T *__restrict__ Cout, int *__restrict__ flag, int zchunk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Fused3DTile<N, T, SF, TX, TY, Q4> t(g, cf, fin, fout, Cin, Cout, flag, smem_raw, zchunk);
    t.march();
}

// Number of z-chunks of a z-marching kernel over `tiles` x/y tiles: the count (1 .. nz / 8)
// that best fills whole waves of `slots` resident CTAs, each chunk paying `warm` planes'
// worth of warm-up work.
inline int zchunks_for(int tiles, int nz, int slots, double warm) {
    int best = 1;
    double best_eff = -1.0;
    const int cmax = max(1, min(nz / 8, 512));
    for (int c = 1; c <= cmax; ++c) {
        const int zc = (nz + c - 1) / c;
        const int cc = (nz + zc - 1) / zc;
        const long long ctas = (long long)tiles * cc;
        const long long waves = (ctas + slots - 1) / slots;
        const double eff = double(ctas) / double(waves * slots) * double(nz) / (double(cc) * (double(zc) + warm));
        if (eff > best_eff + 1e-9) { best_eff = eff; best = cc; }
    }
    return best;
}

// Resident CTAs of `kernel` on the whole GPU (SM count x CTAs per SM at this block and
// shared-memory size).
template <typename K>
inline int resident_ctas(K kernel, int threads, size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 304;
    }
    return max(1, sms * max(1, per_sm));
}

template <int N, typename T, typename SF, int TX, int TY, int Q4>
cudaError_t launch_fused3d(const Geom &g, const Coef<T> &cf, const Buffers &b, int cur, cudaStream_t st) {
    using Sh = Fused3DShape<N, T, TX, TY>;
    static int slots = 0;
    if (!slots) {
        cudaError_t e = cudaFuncSetAttribute(k_fused3d<N, T, SF, TX, TY, Q4>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::BYTES));
        if (e != cudaSuccess) return e;
        slots = resident_ctas(k_fused3d<N, T, SF, TX, TY, Q4>, TX * TY, Sh::BYTES);
    }
    const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    // z-chunks filling whole waves; the warm-up (4 A-planes, 2 B-planes) costs about 2.5 planes
    int chunks = zchunks_for(tiles, g.nz, slots, 2.5);
    const int zchunk = (g.nz + chunks - 1) / chunks;
    chunks = (g.nz + zchunk - 1) / zchunk;
    const dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, chunks);
    k_fused3d<N, T, SF, TX, TY, Q4><<<grid, TX * TY, Sh::BYTES, st>>>(
        g, cf, static_cast<const SF *>(b.f[cur]), static_cast<SF *>(b.f[1 - cur]),
        static_cast<const T *>(b.C[cur]), static_cast<T *>(b.C[1 - cur]), b.flag, zchunk);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Split D3Q19 step: the same site arithmetic as the fused step in two z-marching kernels.
//   k_split3d_phys: per own site, the stencil, force, flux potential and moments (from a
//     shared-memory ring of (C, E_B) on the tile + 1-site ring, staged by cp.async), the TRT
//     collision and push-streaming of f, and v and S written to a scratch array in HBM;
//   k_split3d_gather: per own site, C(t+1) from a shared-memory ring of those records on the
//     tile + 1-site ring (16-byte cp.async copies of the scratch array).
// The scratch array holds per site the gather's record (C, v, S) in TRec planes, |v|^2 being
// formed again after each load, so the gather stages it with 16- and 4-byte copies and reads
// every neighbour with two 16-byte and one 4-byte shared load (N = 4).  The record carries C
// although C(t) is in HBM already: staging C from its own planes takes 4-byte copies into the
// middle of 16-byte records, which meet 4-way shared-memory bank conflicts (measured: the
// gather kernel ran 0.358 instead of 0.27 ms at 256^3).  No site is computed twice (the fused
// step recomputes S and v on the tile's ring), at the cost of the record crossing HBM (write +
// read).  Every value
// is computed by the same device functions in the same order as in the fused step, so both forms
// give the same bits.
// ----------------------------------------------------------------------------
template <int N, typename T, int TX, int TY>
struct Split3DShape {
    static constexpr int RX = TX + 2, RY = TY + 2, PLANE = RX * RY;   // tile + 1-ring
    static constexpr int SLOTS = 4;
    static constexpr int NT = TX * TY;
    static constexpr int ITER = (PLANE + NT - 1) / NT;
    using RA = SRec<T, N>;               // evolved C (N-1), E_B
    using RB = TRec<T, 2 * N + 1>;       // the gather record written to the scratch array
    static constexpr size_t BYTES_A = sizeof(T) * size_t(SLOTS * RA::NVP * PLANE);
};


__device__ __forceinline__ int slot4(int z) { return (z + 8) & 3; }   // z >= -1

// Where one CTA of a split kernel is and which ring sites it stages: a TX x TY tile of sites,
// NT threads (thread t owns site (t % TX, t / TX) when NT = TX * TY).
template <int TX, int TY, int NT, int ITER, int PLANE, int RX>
struct SplitTile {
    int nx, ny, nz, nxy, n, tid, x0, y0, z_lo, z_hi, tx, ty, gx0, gy0, sx, sy, sxy;
    bool edge, wallt, tiny, own_xy;
    int roff[ITER];      // in-plane index (x + nx y) of this thread's ring sites, -1 past the plane

    __device__ __forceinline__ SplitTile(const Geom &g, int zchunk) {
        nx = g.nx; ny = g.ny; nz = g.nz;
        nxy = nx * ny;
        n = int(g.n);
        tid = threadIdx.x;
        x0 = blockIdx.x * TX;
        y0 = blockIdx.y * TY;
        z_lo = blockIdx.z * zchunk;
        z_hi = min(z_lo + zchunk, nz);
        edge = (x0 - 1 < 0) || (x0 + TX + 1 > nx) || (y0 - 1 < 0) || (y0 + TY + 1 > ny);
        wallt = (g.wx && ((x0 - 1 < 0) || (x0 + TX + 1 > nx))) || (g.wy && ((y0 - 1 < 0) || (y0 + TY + 1 > ny)));
        tiny = nx < TX + 2 || ny < TY + 2;
        tx = tid % TX;
        ty = tid / TX;
        gx0 = x0 + tx;
        gy0 = y0 + ty;
        own_xy = gx0 < nx && gy0 < ny;
        sx = edge ? pwrap(gx0, nx, tiny) : gx0;
        sy = edge ? pwrap(gy0, ny, tiny) : gy0;
        sxy = sx + nx * sy;
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int i = tid + it * NT;
            if (i < PLANE) {
                const int ly = i / RX, lx = i - ly * RX;
                int gx = x0 + lx - 1, gy = y0 + ly - 1;
                if (edge) {
                    // periodic wrap; beyond a wall (or a ragged far edge) clamp to a real site:
                    // such entries are never used by a real site
                    gx = g.wx ? min(max(gx, 0), nx - 1) : pwrap(gx, nx, tiny);
                    gy = g.wy ? min(max(gy, 0), ny - 1) : pwrap(gy, ny, tiny);
                }
                roff[it] = gx + nx * gy;
            } else {
                roff[it] = -1;
            }
        }
    }
    __device__ __forceinline__ int zwrap(int z) const { return nz > 1 ? wrap(z, nz) : 0; }
};

// GEO: a geometry of solid and inlet nodes (Sec. III C), given as per-site link masks (k_link_mask)
// with the node classes and the inlet table: links into a solid node take the wall rules (the
// stencil's mirror rule, bounce-back), with the checked forms chosen per warp; links into an
// inlet node take the moving-wall bounce-back of the velocity inlet, while the stencil sees the
// inlet's C_b; a solid or inlet node keeps its f and C and writes the record the gather reads
// from it.
template <int N, typename T, typename SF, int TX, int TY, int Q4, bool GEO = false>
__global__ void __launch_bounds__(TX * TY, (sizeof(T) == 4 ? 512 / (TX * TY) : 256 / (TX * TY)))
k_split3d_phys(Geom g, Coef<T> cf, const SF *__restrict__ fin, SF *__restrict__ fout,
               const T *__restrict__ Cin, T *__restrict__ vs, int zchunk, const unsigned *__restrict__ lmask,
               const unsigned char *__restrict__ node, const T *__restrict__ inl, const T *__restrict__ ghost) {
    using Sh = Split3DShape<N, T, TX, TY>;
    using RA = typename Sh::RA;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sA = reinterpret_cast<T *>(smem_raw);
    constexpr int ASLOT = RA::NVP * Sh::PLANE;
    const SplitTile<TX, TY, Sh::NT, Sh::ITER, Sh::PLANE, Sh::RX> t(g, zchunk);
    const int n = t.n, nz = t.nz;

    // with an outflow, the ring sites beyond x = nx - 1 come from the ghost column: their line
    // (y) index, or -1 for every other ring site
    int grow[Sh::ITER];
#pragma unroll
    for (int it = 0; it < Sh::ITER; ++it) {
        grow[it] = -1;
        if constexpr (GEO) {
            const int i = t.tid + it * Sh::NT;
            if (ghost && i < Sh::PLANE) {
                const int ly = i / Sh::RX, lx = i - ly * Sh::RX;
                if (t.x0 + lx - 1 == t.nx) {
                    const int gy = t.y0 + ly - 1;
                    grow[it] = g.wy ? min(max(gy, 0), t.ny - 1) : pwrap(gy, t.ny, t.tiny);
                }
            }
        }
    }
    // start the copies of the evolved C of plane za (tile + 1-ring), one group
    auto copy_A = [&](int za) {
        if (!(g.wz && (za < 0 || za >= nz))) {
            const int zw = t.zwrap(za);
            const int zo = t.nxy * zw;
            T *base = sA + slot4(za) * ASLOT;
#pragma unroll
            for (int it = 0; it < Sh::ITER; ++it) {
                const int i = t.tid + it * Sh::NT;
                if (t.roff[it] >= 0) {
                    const int rows = t.ny * nz;
#pragma unroll
                    for (int a = 0; a < N - 1; ++a) {
                        const T *src = (GEO && grow[it] >= 0) ? ghost + size_t(a) * rows + (grow[it] + t.ny * zw)
                                                              : Cin + size_t(a) * n + (t.roff[it] + zo);
                        cp_async_value<T>(base + (a / RA::PER) * Sh::PLANE * RA::PER + i * RA::PER + (a % RA::PER), src);
                    }
                }
            }
        }
        cp_async_commit();
    };
    // E_B of this thread's staged sites of plane za (its own copies have landed)
    auto finish_A = [&](int za) {
        if (g.wz && (za < 0 || za >= nz)) return;
        T *base = sA + slot4(za) * ASLOT;
#pragma unroll
        for (int it = 0; it < Sh::ITER; ++it) {
            const int i = t.tid + it * Sh::NT;
            if (t.roff[it] >= 0) {
                T rec[RA::NVP];
                srec_load<T, N>(base, Sh::PLANE, i, rec);
                T cc[N];
                T rest = T(0);
#pragma unroll
                for (int a = 0; a < N - 1; ++a) { cc[a] = rec[a]; rest += rec[a]; }
                cc[N - 1] = T(1) - rest;
                base[((N - 1) / RA::PER) * Sh::PLANE * RA::PER + i * RA::PER + ((N - 1) % RA::PER)] =
                    bulk_energy<N, T>(cc, cf);
            }
        }
    };
    auto load_F = [&](int zb, T (&f)[19]) {
        f[0] = T(0);
        if (!t.own_xy || zb >= t.z_hi) return;
        const int s0 = t.sxy + t.nxy * zb;
        sfor<1, 19, 1>([&](auto kc_) { constexpr int k = decltype(kc_)::value; f[k] = FStore<SF, T>::load(fin + (k - 1) * n + s0, LD3Q19::w(k), cf.finv); });
    };

    T fo[19], fn[19];
    copy_A(t.z_lo - 1);
    copy_A(t.z_lo);
    load_F(t.z_lo, fo);
    cp_async_wait_all();
    finish_A(t.z_lo - 1);
    finish_A(t.z_lo);
    copy_A(t.z_lo + 1);
    // one plane: its site updates with the populations in cur, the next plane's loaded into nxt
    auto plane = [&](int z, T (&cur)[19], T (&nxt)[19]) {
        cp_async_wait_all();
        finish_A(z + 1);
        __syncthreads();                  // A(z-1..z+1) complete; every thread is past plane z-1
        copy_A(z + 2);
        load_F(z + 1, nxt);
        if (t.own_xy) {
            const bool wchk = t.wallt || (g.wz && (z == 0 || z == nz - 1));
            unsigned wall0 = wchk ? wall_mask3(g, t.gx0, t.gy0, z) : 0u;
            const int s0 = t.sxy + t.nxy * z;
            unsigned lm = 0u;
            if constexpr (GEO) {
                lm = lmask[s0];
                wall0 |= lm & kLinkSolidBits;
            }
            const bool check = GEO ? __any_sync(__activemask(), wall0 != 0u || (lm & (kLinkInletNear | kLinkOutflowCol)) != 0u)
                                   : wchk;
            const T *pm = sA + slot4(z - 1) * ASLOT, *p0 = sA + slot4(z) * ASLOT, *pp = sA + slot4(z + 1) * ASLOT;
            const int ia = (t.ty + 1) * Sh::RX + (t.tx + 1);
            T c[N], lap[N], gr[N][3], gE[3];
            if (check) stencil3d<N, T, Sh::RX, true>(pm, p0, pp, Sh::PLANE, ia, wall0, c, lap, gr, gE);
            else       stencil3d<N, T, Sh::RX, false>(pm, p0, pp, Sh::PLANE, ia, 0u, c, lap, gr, gE);
            if (GEO && (lm & kLinkNonFluid)) {
                // a solid or inlet node keeps its state: f copied as stored; its record is (C, 0, 0)
                // for a solid node (the gather copies C back out) and the prescribed state
                // (C_b, v_b, S_b) for an inlet node (the gather's terms from it carry g^eq of that
                // state, and its own C stays C_b)
                T rec[2 * N + 1];
                const unsigned cls = link_class(lm);
                if (cls >= kNodeInlet0) {
                    const T *row = inl + (cls - kNodeInlet0) * (2 * N + 1);
#pragma unroll
                    for (int a = 0; a < N - 1; ++a) { rec[a] = row[3 + a]; rec[N + 2 + a] = row[N + 2 + a]; }
                    rec[N - 1] = row[0]; rec[N] = row[1]; rec[N + 1] = row[2];
                } else {
#pragma unroll
                    for (int a = 0; a < 2 * N + 1; ++a) rec[a] = a < N - 1 ? c[a] : T(0);
                }
                trec_store<T, 2 * N + 1>(vs, size_t(n), size_t(s0), rec);
#pragma unroll
                for (int k = 1; k < 19; ++k) fout[size_t(k - 1) * n + s0] = fin[size_t(k - 1) * n + s0];
                return;
            }
            T S[N - 1], F[3], v[3], P, sp[9], dm[9];
            site_physics3d<N, T, Q4>(cf, c, lap, gr, gE, cur, S, F, v, P, sp, dm);
            {
                // the gather record (C, v, S) of this site, TRec planes over the grid
                T rec[2 * N + 1];
#pragma unroll
                for (int a = 0; a < N - 1; ++a) { rec[a] = c[a]; rec[N + 2 + a] = S[a]; }
                rec[N - 1] = v[0]; rec[N] = v[1]; rec[N + 1] = v[2];
                trec_store<T, 2 * N + 1>(vs, size_t(n), size_t(s0), rec);
            }
            collide3d<N, T>(cf, c, v, F, P, sp, dm, cur);
            if constexpr (GEO) {
                if (lm & kLinkInletNear) {
                    // links into an inlet node (Sec. III C, velocity inlet): the population that
                    // would enter it comes back as f*_k(x) - 6 w_k e_k . v_b into direction kbar
                    const int nxy = t.nx * t.ny;
                    sfor<1, 19, 1>([&](auto kc_) {
                        constexpr int k = decltype(kc_)::value;
                        constexpr int ex = LD3Q19::ex(k), ey = LD3Q19::ey(k), ez = LD3Q19::ez(k);
                        if ((wall0 >> k) & 1u) return;      // beyond a wall or solid: plain bounce-back
                        const int xx = t.sx + ex, yy = t.sy + ey, zz = z + ez;
                        const int xw = xx < 0 ? xx + t.nx : (xx >= t.nx ? xx - t.nx : xx);
                        const int yw = yy < 0 ? yy + t.ny : (yy >= t.ny ? yy - t.ny : yy);
                        const int zw = zz < 0 ? zz + nz : (zz >= nz ? zz - nz : zz);
                        const unsigned char cls = node[xw + t.nx * yw + nxy * zw];
                        if (cls >= kNodeInlet0) {
                            const T *row = inl + (cls - kNodeInlet0) * (2 * N + 1);
                            const T eu = T(ex) * row[0] + T(ey) * row[1] + T(ez) * row[2];
                            cur[k] -= T(6.0 * LD3Q19::w(k)) * eu;
                            wall0 |= 1u << k;
                        }
                    });
                }
            }
            // with an outflow, the links of column nx - 1 into the ghost column are dropped (the
            // convective condition then replaces that column's populations)
            const unsigned drop = (GEO && (lm & kLinkOutflowCol)) ? d3q19_xplus_mask() : 0u;
            push_store3d<T, SF>(cf, fout, n, t.nx, t.ny, nz, t.sx, t.sy, z, s0, wall0, cur, GEO && check, drop);
        }
    };
    // one plane per iteration (two per iteration with the population registers swapping roles
    // doubles the loop body and measured slower)
#pragma unroll 1
    for (int z = t.z_lo; z < t.z_hi; ++z) {
        plane(z, fo, fn);
#pragma unroll
        for (int k = 0; k < 19; ++k) fo[k] = fn[k];
    }
    cp_async_wait_all();                  // no copy outlives the CTA
}

// Shape of the gather kernel: TX x (SPT TYT) sites, TX x TYT threads, SPT sites stacked in y each.
template <int N, typename T, int TX, int TYT, int SPT>
struct Gather3DShape {
    static constexpr int TY = SPT * TYT;
    static constexpr int RX = TX + 2, RY = TY + 2, PLANE = RX * RY;   // tile + 1-ring
    static constexpr int SLOTS = 4;
    static constexpr int NT = TX * TYT;
    static constexpr int ITER = (PLANE + NT - 1) / NT;
    using RB = TRec<T, 2 * N + 1>;       // the gather record without |v|^2
    static constexpr size_t BYTES = sizeof(T) * size_t(SLOTS * RB::NVP * PLANE);
};

// SF (the storage type of f, unused here) keeps the instantiations of the FP32, FP16 and BF16
// translation units apart: each sets the shared-memory attribute of the kernel it launches.
// TAUG: stored component populations (tau_g != 1), each of the thread's sites on its own.
// GEO: a geometry of solid and inlet nodes (link masks as for the physics kernel): a source
// inside a solid node bounces back, with the checked form chosen per warp; a source at an inlet
// node contributes g^eq of the inlet's prescribed state through its record; a solid or inlet
// node keeps its C.
template <int N, typename T, typename SF, int TX, int TYT, int SPT, bool TAUG, bool GEO = false>
__global__ void __launch_bounds__(TX * TYT, (sizeof(T) == 4 ? 512 / (TX * TYT) : 256 / (TX * TYT)))
k_split3d_gather(Geom g, T m, T omg, const T *__restrict__ vs, T *__restrict__ Cout, int *__restrict__ flag, int zchunk,
                 const T *__restrict__ gin, T *__restrict__ gout, const unsigned *__restrict__ lmask) {
    using Sh = Gather3DShape<N, T, TX, TYT, SPT>;
    using RB = typename Sh::RB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sB = reinterpret_cast<T *>(smem_raw);
    constexpr int BSLOT = RB::NVP * Sh::PLANE;
    const SplitTile<TX, Sh::TY, Sh::NT, Sh::ITER, Sh::PLANE, Sh::RX> t(g, zchunk);
    const int n = t.n, nz = t.nz, nx = t.nx, ny = t.ny;
    // this thread's sites: column tx, rows SPT r .. SPT r + SPT - 1 of the tile
    const int tx = t.tid % TX, tr = t.tid / TX;
    const int gx = t.x0 + tx, gy0 = t.y0 + SPT * tr;
    const int sx = t.edge ? pwrap(gx, nx, t.tiny) : gx;
    int sy[SPT];
    bool own[SPT];
#pragma unroll
    for (int j = 0; j < SPT; ++j) {
        own[j] = gx < nx && gy0 + j < ny;
        sy[j] = t.edge ? pwrap(gy0 + j, ny, t.tiny) : gy0 + j;
    }
    // start the copies of the records of plane zb (tile + 1-ring), one group
    auto copy_B = [&](int zb) {
        if (!(g.wz && (zb < 0 || zb >= nz))) {
            const int zo = t.nxy * t.zwrap(zb);
            T *base = sB + slot4(zb) * BSLOT;
#pragma unroll
            for (int it = 0; it < Sh::ITER; ++it) {
                const int i = t.tid + it * Sh::NT;
                if (t.roff[it] >= 0) {
                    const int s = t.roff[it] + zo;
#pragma unroll
                    for (int ch = 0; ch < RB::NC; ++ch) {
                        const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(base + RB::chunk_at(ch, Sh::PLANE) + size_t(i) * RB::PER));
                        const T *src = vs + RB::chunk_at(ch, size_t(n)) + size_t(s) * RB::PER;
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
                    }
                    if constexpr (RB::TAIL2 == 2) {
                        const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(base + RB::tail2_at(Sh::PLANE) + size_t(i) * 2));
                        const T *src = vs + RB::tail2_at(size_t(n)) + size_t(s) * 2;
                        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
                    }
                    if constexpr (RB::TAIL1 == 1) {
                        cp_async_value<T>(base + RB::tail1_at(Sh::PLANE) + i, vs + RB::tail1_at(size_t(n)) + s);
                    }
                }
            }
        }
        cp_async_commit();
    };

    copy_B(t.z_lo - 1);
    copy_B(t.z_lo);
    copy_B(t.z_lo + 1);
#pragma unroll 1
    for (int z = t.z_lo; z < t.z_hi; ++z) {
        cp_async_wait_all();
        __syncthreads();                  // B(z-1..z+1) complete; every thread is past plane z-1
        copy_B(z + 2);
        if (own[0]) {
            const bool check = t.wallt || (g.wz && (z == 0 || z == nz - 1));
            unsigned wall[SPT];
            unsigned wany = 0u;
#pragma unroll
            for (int j = 0; j < SPT; ++j) {
                wall[j] = check && own[j] ? wall_mask3(g, gx, gy0 + j, z) : 0u;
                if constexpr (GEO)
                    if (own[j]) wall[j] |= lmask[sx + nx * sy[j] + t.nxy * z] & kLinkSolidBits;
                wany |= wall[j];
            }
            if constexpr (GEO) wany = __any_sync(__activemask(), wany != 0u) ? 1u : 0u;
            const T *bm = sB + slot4(z - 1) * BSLOT, *b0 = sB + slot4(z) * BSLOT, *bp = sB + slot4(z + 1) * BSLOT;
            const int ib = (SPT * tr + 1) * Sh::RX + (tx + 1);
            T out[SPT][N - 1];
            if constexpr (TAUG) {
#pragma unroll
                for (int j = 0; j < SPT; ++j) {
                    if (!own[j]) continue;
                    const int sj = sx + nx * sy[j] + t.nxy * z;
                    if (wall[j]) gather3d_taug<N, T, Sh::RX, true, true>(bm, b0, bp, Sh::PLANE, ib + j * Sh::RX, wall[j], m, omg, gin, gout, n, nx, ny, nz, sx, sy[j], z, sj, out[j]);
                    else         gather3d_taug<N, T, Sh::RX, false, true>(bm, b0, bp, Sh::PLANE, ib + j * Sh::RX, 0u, m, omg, gin, gout, n, nx, ny, nz, sx, sy[j], z, sj, out[j]);
                }
            } else {
                // the wall-free form carries no bounce-back code; the form is decided per thread
                if (wany) gather3d_stack<N, T, Sh::RX, true, true, SPT>(bm, b0, bp, Sh::PLANE, ib, wall, m, out);
                else      gather3d_stack<N, T, Sh::RX, false, true, SPT>(bm, b0, bp, Sh::PLANE, ib, wall, m, out);
            }
            if constexpr (GEO) {
                // a solid or inlet node keeps its C (the first values of its record)
#pragma unroll
                for (int j = 0; j < SPT; ++j) {
                    if (!own[j] || (lmask[sx + nx * sy[j] + t.nxy * z] & kLinkNonFluid) == 0u) continue;
                    T r[RB::NVP + 1];
                    BRec<T, 2 * N + 2, true>::load(b0, Sh::PLANE, ib + j * Sh::RX, r);
#pragma unroll
                    for (int e = 0; e < N - 1; ++e) out[j][e] = r[e];
                }
            }
            bool bad = false;
#pragma unroll
            for (int j = 0; j < SPT; ++j) {
                if (!own[j]) continue;
                const int sj = sx + nx * sy[j] + t.nxy * z;
#pragma unroll
                for (int e = 0; e < N - 1; ++e) {
                    Cout[size_t(e) * n + sj] = out[j][e];
                    bad |= !isfinite(out[j][e]);
                }
            }
            if (bad) atomicOr(flag, 1);
        }
    }
    cp_async_wait_all();                  // no copy outlives the CTA
}

// z-chunks of a split kernel filling whole waves of `slots` resident CTAs (the warm-up of a
// chunk, two staged planes, costs about half a plane of work)
inline dim3 split3d_grid(const Geom &g, int TX, int TY, int slots, int &zchunk) {
    const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    int chunks = zchunks_for(tiles, g.nz, slots, 0.5);
    zchunk = (g.nz + chunks - 1) / chunks;
    chunks = (g.nz + zchunk - 1) / zchunk;
    return dim3((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, chunks);
}

template <int N, typename T, typename SF, int TX, int TY, int Q4, bool GEO = false>
cudaError_t launch_split3d_phys(const Geom &g, const Coef<T> &cf, const Buffers &b, int cur, cudaStream_t st) {
    using Sh = Split3DShape<N, T, TX, TY>;
    static int slots = 0;
    if (!slots) {
        cudaError_t e = cudaFuncSetAttribute(k_split3d_phys<N, T, SF, TX, TY, Q4, GEO>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::BYTES_A));
        if (e != cudaSuccess) return e;
        slots = resident_ctas(k_split3d_phys<N, T, SF, TX, TY, Q4, GEO>, TX * TY, Sh::BYTES_A);
    }
    int zchunk = 0;
    const dim3 grid = split3d_grid(g, TX, TY, slots, zchunk);
    k_split3d_phys<N, T, SF, TX, TY, Q4, GEO><<<grid, TX * TY, Sh::BYTES_A, st>>>(
        g, cf, static_cast<const SF *>(b.f[cur]), static_cast<SF *>(b.f[1 - cur]), static_cast<const T *>(b.C[cur]),
        static_cast<T *>(b.vs), zchunk, GEO ? b.lmask : nullptr, GEO ? b.node : nullptr,
        GEO ? static_cast<const T *>(b.inl) : nullptr,
        (GEO && b.outflow) ? static_cast<const T *>(b.ghost[cur]) : nullptr);
    return cudaGetLastError();
}

template <int N, typename T, typename SF, int TX, int TYT, int SPT, bool TAUG, bool GEO = false>
cudaError_t launch_split3d_gather(const Geom &g, const Coef<T> &cf, const Buffers &b, int cur, cudaStream_t st) {
    using Sh = Gather3DShape<N, T, TX, TYT, SPT>;
    static int slots = 0;
    if (!slots) {
        cudaError_t e = cudaFuncSetAttribute(k_split3d_gather<N, T, SF, TX, TYT, SPT, TAUG, GEO>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::BYTES));
        if (e != cudaSuccess) return e;
        slots = resident_ctas(k_split3d_gather<N, T, SF, TX, TYT, SPT, TAUG, GEO>, TX * TYT, Sh::BYTES);
    }
    int zchunk = 0;
    const dim3 grid = split3d_grid(g, TX, Sh::TY, slots, zchunk);
    k_split3d_gather<N, T, SF, TX, TYT, SPT, TAUG, GEO><<<grid, TX * TYT, Sh::BYTES, st>>>(
        g, cf.m, cf.gomega, static_cast<const T *>(b.vs), static_cast<T *>(b.C[1 - cur]), b.flag, zchunk,
        static_cast<const T *>(b.g[cur]), static_cast<T *>(b.g[1 - cur]), GEO ? b.lmask : nullptr);
    return cudaGetLastError();
}

// D3Q19 dispatch.  Variants 0, 1: the fused step (32 x 4, 32 x 8; the wider one only where its
// rings fit the 227 KB of shared memory of a CTA).  Variants 2, 3: the split step (32 x 8, 32 x 4),
// two kernels per step (kern[0]: physics and streaming, kern[1]: the Cahn-Hilliard gather).
template <int N, typename T, typename SF>
struct Fused3DLaunch {
    // the fused form is built for N <= 4 only (the split form is faster at every measured size and
    // its instantiations for N = 5..8 would double the build); there variants 0 and 1 alias 3 and 2
    static constexpr bool kFused = N <= 4;
    static constexpr bool kWideFits = Fused3DShape<N, T, 32, 8>::BYTES <= 220 * 1024;
    template <int TYT, int SPT> static constexpr bool gather_fits = Gather3DShape<N, T, 32, TYT, SPT>::BYTES <= 220 * 1024;
    // sites per gather thread: three where the three sites' records and sums stay in registers
    static constexpr int kSpt = (sizeof(T) == 4 && N <= 4) ? 3 : 2;
    static constexpr int kGatherLarge = gather_fits<8, 2> ? 8 : (gather_fits<4, 2> ? 4 : 2);
    static constexpr int kGatherSmall = gather_fits<4, 2> ? 4 : 2;
    static constexpr int kGatherStack = gather_fits<4, kSpt> ? 4 : (gather_fits<2, kSpt> ? 2 : 1);
    static_assert(gather_fits<2, 2> && gather_fits<1, kSpt>, "the smallest gather tiles fit");
    static cudaError_t step(const Geom &g, const void *coef, const Buffers &b, int cur, cudaStream_t st, int variant) {
        const Coef<T> &cf = *static_cast<const Coef<T> *>(coef);
        // a geometry of solid and inlet nodes: the split form's geometry kernels, one tile shape
        if (b.node) return launch_split3d_phys<N, T, SF, 32, 4, Q4_PARAM, true>(g, cf, b, cur, st);
        // the no-phi ablation (flux potential of Eq. 12 without phi_j) and the stored component
        // populations (tau_g != 1) run in the split form only: every variant launches its physics
        // kernel
        if (cf.no_phi || b.g[0]) {
            if (!cf.no_phi) {
                if (variant == 3 || variant == 0) return launch_split3d_phys<N, T, SF, 32, 4, Q4_PARAM>(g, cf, b, cur, st);
                return launch_split3d_phys<N, T, SF, 32, 8, Q4_PARAM>(g, cf, b, cur, st);
            }
            if (variant == 3 || variant == 0) return launch_split3d_phys<N, T, SF, 32, 4, Q4_NOPHI>(g, cf, b, cur, st);
            return launch_split3d_phys<N, T, SF, 32, 8, Q4_NOPHI>(g, cf, b, cur, st);
        }
        if constexpr (!kFused) {
            if (variant < 2) variant = variant == 0 ? 3 : 2;
        }
        if (variant == 2) return launch_split3d_phys<N, T, SF, 32, 8, Q4_PARAM>(g, cf, b, cur, st);
        if (variant == 3) return launch_split3d_phys<N, T, SF, 32, 4, Q4_PARAM>(g, cf, b, cur, st);
        if constexpr (kFused) {
            if constexpr (kWideFits) {
                if (variant == 1) return launch_fused3d<N, T, SF, 32, 8, Q4_PARAM>(g, cf, b, cur, st);
            }
            return launch_fused3d<N, T, SF, 32, 4, Q4_PARAM>(g, cf, b, cur, st);
        }
        return cudaErrorInvalidValue;
    }
    static cudaError_t gather(const Geom &g, const void *coef, const Buffers &b, int cur, cudaStream_t st, int variant) {
        const Coef<T> &cf = *static_cast<const Coef<T> *>(coef);
        if (cf.no_phi || b.g[0] || !kFused) variant = (variant == 3 || variant == 0) ? 3 : 2;
        if (b.node) {
            cudaError_t e = launch_split3d_gather<N, T, SF, 32, kGatherSmall, 2, false, true>(g, cf, b, cur, st);
            if (e == cudaSuccess && b.outflow) e = launch_outflow<LD3Q19, N, T, SF>(g, cf, b, cur, st);
            return e;
        }
        // stored component populations (tau_g != 1): one tile shape
        if (b.g[0]) return launch_split3d_gather<N, T, SF, 32, kGatherSmall, 2, true>(g, cf, b, cur, st);
        // variant 3: kSpt sites per thread on 32 x 4 threads (32 x 12 sites for FP32, N <= 4, else
        // 32 x 8); variant 2: two sites per thread, 32 x 16 sites on 256 threads; each with the next
        // smaller tile where its four record planes do not fit a CTA's shared memory
        if (variant == 3) return launch_split3d_gather<N, T, SF, 32, kGatherStack, kSpt, false>(g, cf, b, cur, st);
        return launch_split3d_gather<N, T, SF, 32, kGatherLarge, 2, false>(g, cf, b, cur, st);
    }
    static const Ops *ops(int prec) {
        using B = Launch<LD3Q19, N, T, SF>;
        static const Ops o = {19, 3, N, prec, 1, {K_FUSED, K_FUSED}, {&step, &gather}, 4,
                              {kFused ? "fused3d 32x4" : "split3d 32x4", kFused ? "fused3d 32x8" : "split3d 32x8",
                               "split3d 32x8", "split3d 32x4"},
                              &B::moments, &B::reduce, &B::init_f, &B::unpack_f, &B::pack_C, &B::init_g,
                              int(sizeof(SF)), int(sizeof(T)), &B::inlet_table3, &B::prepare_solid, &B::moments_solid,
                              {kFused ? 1 : 2, kFused ? 1 : 2, 2, 2},
                              {{kFused ? K_FUSED : K_PHYS, kFused ? K_FUSED : K_GATHER},
                               {kFused ? K_FUSED : K_PHYS, kFused ? K_FUSED : K_GATHER}, {K_PHYS, K_GATHER}, {K_PHYS, K_GATHER}},
                              TRec<T, 2 * N + 1>::NVP};
        return &o;
    }
};

// One component count per call; the translation units instantiate a few counts each, so that the
// build compiles them in parallel.
template <int NN, typename T, typename SF>
const Ops *ops_fused3d_one(int prec) { return Fused3DLaunch<NN, T, SF>::ops(prec); }

}  // namespace nfe
