// Fused D3Q19 time step: one kernel per step.  A CTA owns a TX x TY column of
// the grid over a chunk of z-planes and marches up in z with shared-memory
// ring buffers:
//   A ring (5 planes, tile + 2-site ring in x/y): evolved C and the bulk energy
//     E_B (Eq. 5), computed once per site;
//   B ring (3 planes, tile + 1-site ring): evolved C, v and the flux potential S.
// For every plane z of the chunk the CTA
//   1. fills A-plane z+2 from HBM,
//   2. computes B-plane z+1: isotropic grad / Laplacian (Eqs. 35-36) from A-planes
//      z..z+2, S_i = C_i q_i(C) + (3D/4) lap C_i (Eq. 12), the force of Eq. 34,
//      moments of f (Eqs. 37-38); the own sites of plane z+1 are collided (TRT with
//      forcing, Eqs. 23-30) and push-streamed with bounce-back (Eqs. 44-45),
//   3. computes C(t+1) of plane z from B-planes z-1..z+1 (Eqs. 39-41, tau_g = 1).
// Only f (18 populations) and the N-1 evolved C cross HBM; the redundant work is
// the x/y ring only, the z direction is streamed.
#pragma once

#include "nfe_fused2d.cuh"

namespace nfe {

template <int N, typename T, int TX, int TY>
struct Fused3DShape {
    static constexpr int AX = TX + 4, AY = TY + 4, APLANE = AX * AY;
    static constexpr int BX = TX + 2, BY = TY + 2, BPLANE = BX * BY;
    using RA = SRec<T, N>;               // evolved C (N-1), E_B
    using RB = SRec<T, 2 * N + 2>;       // evolved C (N-1), vx, vy, vz, S (N-1), |v|^2
    static constexpr int A_SLOT = RA::NVP * APLANE;
    static constexpr int B_SLOT = RB::NVP * BPLANE;
    static constexpr size_t BYTES = sizeof(T) * size_t(5 * A_SLOT + 3 * B_SLOT);
    static constexpr int NHALO = BPLANE - TX * TY;
};

__device__ __forceinline__ int slotA(int z) { return (z + 10) % 5; }   // z >= -2
__device__ __forceinline__ int slotB(int z) { return (z + 9) % 3; }    // z >= -1

// 3-D stencil from three A-planes (below, centre, above) at in-plane index ia.
template <int N, typename T, int AX, bool CHECK>
__device__ __forceinline__ void stencil3d(const T *pm, const T *p0, const T *pp, int count, int ia, unsigned wall,
                                          T (&c)[N], T (&lap)[N], T (&g)[N][3], T (&gE)[3]) {
    using RA = SRec<T, N>;
    T r0[RA::NVP];
    srec_load<T, N>(p0, count, ia, r0);
    T acc[N][4];          // lap, gx, gy, gz sums (N-1 = bulk energy: gradient only)
#pragma unroll
    for (int a = 0; a < N; ++a) acc[a][0] = acc[a][1] = acc[a][2] = acc[a][3] = T(0);
    sfor<1, 19, 1>([&](auto kc_) {
        constexpr int k = decltype(kc_)::value;
        if (CHECK && ((wall >> k) & 1u)) return;     // psi beyond a wall := psi(x)
        const T *pl = LD3Q19::ez(k) > 0 ? pp : (LD3Q19::ez(k) < 0 ? pm : p0);
        T r[RA::NVP];
        srec_load<T, N>(pl, count, ia + LD3Q19::ex(k) + AX * LD3Q19::ey(k), r);
        const T wk = T(LD3Q19::w(k));
#pragma unroll
        for (int a = 0; a < N; ++a) {
            const T d = r[a] - r0[a];
            if (a < N - 1) acc[a][0] += wk * d;
            if (LD3Q19::ex(k)) acc[a][1] += (LD3Q19::ex(k) > 0 ? wk : -wk) * d;
            if (LD3Q19::ey(k)) acc[a][2] += (LD3Q19::ey(k) > 0 ? wk : -wk) * d;
            if (LD3Q19::ez(k)) acc[a][3] += (LD3Q19::ez(k) > 0 ? wk : -wk) * d;
        }
    });
    T sl = T(0), sx = T(0), sy = T(0), sz = T(0), rest = T(0);
#pragma unroll
    for (int a = 0; a < N - 1; ++a) {
        c[a] = r0[a];
        rest += r0[a];
        lap[a] = T(6) * acc[a][0];
        g[a][0] = T(3) * acc[a][1]; g[a][1] = T(3) * acc[a][2]; g[a][2] = T(3) * acc[a][3];
        sl += lap[a]; sx += g[a][0]; sy += g[a][1]; sz += g[a][2];
    }
    c[N - 1] = T(1) - rest;
    lap[N - 1] = -sl; g[N - 1][0] = -sx; g[N - 1][1] = -sy; g[N - 1][2] = -sz;
    gE[0] = T(3) * acc[N - 1][1]; gE[1] = T(3) * acc[N - 1][2]; gE[2] = T(3) * acc[N - 1][3];
}

template <int N, typename T, int Q4>
__device__ __forceinline__ void site_physics3d(const Coef<T> &cf, const T (&c)[N], const T (&lap)[N],
                                               const T (&g)[N][3], const T (&gE)[3], const T (&f)[19],
                                               T (&S)[N - 1], T (&F)[3], T (&v)[3], T &P) {
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
    T j0 = T(0), j1 = T(0), j2 = T(0), sumf = T(0);
    sfor<1, 19, 1>([&](auto kc_) {
        constexpr int k = decltype(kc_)::value;
        sumf += f[k];
        if (LD3Q19::ex(k)) j0 += LD3Q19::ex(k) > 0 ? f[k] : -f[k];
        if (LD3Q19::ey(k)) j1 += LD3Q19::ey(k) > 0 ? f[k] : -f[k];
        if (LD3Q19::ez(k)) j2 += LD3Q19::ez(k) > 0 ? f[k] : -f[k];
    });
    v[0] = j0 + T(0.5) * F[0];
    v[1] = j1 + T(0.5) * F[1];
    v[2] = j2 + T(0.5) * F[2];
    const T w0 = T(1) / T(3);
    P = (sumf - T(1.5) * w0 * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2])) * T(1.0 / (3.0 * (1.0 - 1.0 / 3.0)));
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

    __device__ __forceinline__ Fused3DTile(const Geom &g_, const Coef<T> &cf_, const SF *fin_, SF *fout_,
                                           const T *Cin_, T *Cout_, int *flag_, unsigned char *smem, int zchunk)
        : g(g_), cf(cf_), fin(fin_), fout(fout_), Cin(Cin_), Cout(Cout_), flag(flag_) {
        sA = reinterpret_cast<T *>(smem);
        sB = sA + 5 * Sh::A_SLOT;
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
    }

    // Periodic plane index of z in [z_lo - 2, z_hi + 2) without a division.
    __device__ __forceinline__ int zwrap(int z) const { return nz > 1 ? wrap(z, nz) : 0; }

    // Loads are issued one plane ahead (load_A / load_F) and consumed by fill_A /
    // fill_B in the next iteration, so HBM latency overlaps the previous plane's work.
    // load_A / fill_A: A-plane za (C and E_B on the tile + 2-ring).
    // load_F: f of the own site and of the ring site of plane zb.
    // fill_B: B-plane zb (S, v; for own planes also collide + push-stream).
    // ch: Cahn-Hilliard update of plane zc from B-planes zc-1..zc+1.
    __device__ __forceinline__ void load_A(int za, T (&cl)[ITER][N - 1]) {
        if (g.wz && (za < 0 || za >= nz)) return;
        const int zw = zwrap(za);
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
                const int s = gx + nx * gy + nxy * zw;
#pragma unroll
                for (int a = 0; a < N - 1; ++a) cl[it][a] = Cin[a * n + s];
            }
        }
    }

    __device__ __forceinline__ void fill_A(int za, const T (&cl)[ITER][N - 1]) {
        if (g.wz && (za < 0 || za >= nz)) return;      // beyond a wall: never read
        T *base = sA + slotA(za) * Sh::A_SLOT;
#pragma unroll
        for (int it = 0; it < ITER; ++it) {
            const int i = tid + it * NT;
            if (i < Sh::APLANE) {
                T rec[RA::NVP];
                T cc[N];
                T rest = T(0);
#pragma unroll
                for (int a = 0; a < N - 1; ++a) { cc[a] = cl[it][a]; rec[a] = cc[a]; rest += cc[a]; }
                cc[N - 1] = T(1) - rest;
                rec[N - 1] = bulk_energy<N, T>(cc, cf);
#pragma unroll
                for (int a = N; a < RA::NVP; ++a) rec[a] = T(0);
                srec_store<T, N>(base, Sh::APLANE, i, rec);
            }
        }
    }

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
            T S[N - 1], F[3], v[3], P;
            site_physics3d<N, T, Q4>(cf, c, lap, gr, gE, f, S, F, v, P);
            T rec[RB::NVP];
#pragma unroll
            for (int a = 0; a < N - 1; ++a) { rec[a] = c[a]; rec[N + 2 + a] = S[a]; }
            rec[N - 1] = v[0]; rec[N] = v[1]; rec[N + 1] = v[2];
            rec[2 * N + 1] = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];   // read 18 times by the gather
#pragma unroll
            for (int a = 2 * N + 2; a < RB::NVP; ++a) rec[a] = T(0);
            srec_store<T, 2 * N + 2>(bbase, Sh::BPLANE, (ty + 1) * Sh::BX + (tx + 1), rec);
            if (collide && own_xy) {
                T op, om;
                relaxation<N, T>(cf, c, op, om);
                const T ap = T(1) - T(0.5) * op, am = T(1) - T(0.5) * om;
                const T vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
                const T vF = v[0] * F[0] + v[1] * F[1] + v[2] * F[2];
                const T base = T(3) * P - T(1.5) * vv;
                // TRT with forcing (Eqs. 23-30) regrouped so that per-site factors are formed once:
                // for a pair (k, kbar), with s = f_k + f_kbar and d = f_k - f_kbar,
                //   sym  = w_k [X + e.v (Y e.v + Z e.F)] - (op / 2) s
                //   anti = w_k (U e.v + V e.F) - (om / 2) d
                // where X = op (3P - 1.5 v.v) - 3 ap v.F, Y = 4.5 op, Z = 9 ap, U = 3 om, V = 3 am;
                // w_k X ... w_k V are shared by all pairs of one weight class.
                const T hop = T(0.5) * op, hom = T(0.5) * om;
                const T X = op * base - T(3) * ap * vF, Y = T(4.5) * op, Z = T(9) * ap, U = T(3) * om, V = T(3) * am;
                // no wrap and no wall for any target: the site is inside the domain by one site
                const bool fast = sx > 0 && sx < nx - 1 && sy > 0 && sy < ny - 1 && zw > 0 && zw < nz - 1;
                sfor<1, 19, 2>([&](auto kc_) {
                    constexpr int k = decltype(kc_)::value;
                    const int kb = k + 1;
                    const T wk = T(LD3Q19::w(k));
                    const T eu = T(LD3Q19::ex(k)) * v[0] + T(LD3Q19::ey(k)) * v[1] + T(LD3Q19::ez(k)) * v[2];
                    const T eF = T(LD3Q19::ex(k)) * F[0] + T(LD3Q19::ey(k)) * F[1] + T(LD3Q19::ez(k)) * F[2];
                    const T sp = f[k] + f[kb], dm = f[k] - f[kb];
                    const T sym = (wk * X + eu * ((wk * Y) * eu + (wk * Z) * eF)) - hop * sp;
                    const T anti = ((wk * U) * eu + (wk * V) * eF) - hom * dm;
                    // post-collision values replace f in place (each pair is read once)
                    f[k] = f[k] + sym + anti;
                    f[kb] = f[kb] + sym - anti;
                });
                // one branch around the whole store block: inside the unrolled loop the
                // compiler would predicate both forms for every site
                if (fast) {
                    sfor<1, 19, 1>([&](auto kc_) {
                        constexpr int k = decltype(kc_)::value;
                        constexpr int dk0 = LD3Q19::ex(k);
                        const int dk = dk0 + nx * LD3Q19::ey(k) + nxy * LD3Q19::ez(k);
                        FStore<SF, T>::store(fout + (k - 1) * n + (s0 + dk), f[k], LD3Q19::w(k), cf.fscale);
                    });
                } else {
                    sfor<1, 19, 1>([&](auto kc_) {
                        constexpr int k = decltype(kc_)::value;
                        constexpr int kb = opp(k);
                        if ((wall0 >> k) & 1u) {
                            // halfway bounce-back: f_kbar(x, t+1) = post_k(x)
                            FStore<SF, T>::store(fout + (kb - 1) * n + s0, f[k], LD3Q19::w(kb), cf.fscale);
                        } else {
                            const int t = wrap(sx + LD3Q19::ex(k), nx) + nx * wrap(sy + LD3Q19::ey(k), ny) +
                                          nxy * wrap(zw + LD3Q19::ez(k), nz);
                            FStore<SF, T>::store(fout + (k - 1) * n + t, f[k], LD3Q19::w(k), cf.fscale);
                        }
                    });
                }
            }
        }
        // ring site
        if (ring_xy_ok) {
            const T (&f)[19] = fr;
            const unsigned wall = check ? wall_mask3(g, hx, hy, zb) : 0u;
            T c[N], lap[N], gr[N][3], gE[3];
            const int ia = (by + 1) * Sh::AX + (bx + 1);
            if (check) stencil3d<N, T, Sh::AX, true>(pm, p0, pp, Sh::APLANE, ia, wall, c, lap, gr, gE);
            else       stencil3d<N, T, Sh::AX, false>(pm, p0, pp, Sh::APLANE, ia, 0u, c, lap, gr, gE);
            T S[N - 1], F[3], v[3], P;
            site_physics3d<N, T, Q4>(cf, c, lap, gr, gE, f, S, F, v, P);
            T rec[RB::NVP];
#pragma unroll
            for (int a = 0; a < N - 1; ++a) { rec[a] = c[a]; rec[N + 2 + a] = S[a]; }
            rec[N - 1] = v[0]; rec[N] = v[1]; rec[N + 1] = v[2];
            rec[2 * N + 1] = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
#pragma unroll
            for (int a = 2 * N + 2; a < RB::NVP; ++a) rec[a] = T(0);
            srec_store<T, 2 * N + 2>(bbase, Sh::BPLANE, by * Sh::BX + bx, rec);
        }
    }

    template <bool CHECK>
    __device__ __forceinline__ void ch_impl(int zc, unsigned wall0) {
        const T *bm = sB + slotB(zc - 1) * Sh::B_SLOT;
        const T *b0 = sB + slotB(zc) * Sh::B_SLOT;
        const T *bp = sB + slotB(zc + 1) * Sh::B_SLOT;
        const int ib = (ty + 1) * Sh::BX + (tx + 1);
        T r0[RB::NVP];
        srec_load<T, 2 * N + 2>(b0, Sh::BPLANE, ib, r0);
        const T vv0 = r0[2 * N + 1];
        const T w0 = T(1) / T(3);
        T acc[N - 1], lapS[N - 1];
#pragma unroll
        for (int e = 0; e < N - 1; ++e) { acc[e] = r0[e] * (-T(1.5) * w0 * vv0); lapS[e] = T(0); }   // increments only
        sfor<1, 19, 1>([&](auto kc_) {
            constexpr int k = decltype(kc_)::value;
            const T wk = T(LD3Q19::w(k));
            const int kb = opp(k);                  // source x - e_k = x + e_kbar
            if (CHECK && ((wall0 >> kb) & 1u)) {
                const T eu = -(T(LD3Q19::ex(k)) * r0[N - 1] + T(LD3Q19::ey(k)) * r0[N] + T(LD3Q19::ez(k)) * r0[N + 1]);
                const T sk = wk * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * vv0);
#pragma unroll
                for (int e = 0; e < N - 1; ++e) acc[e] += r0[e] * sk;      // S difference is zero
            } else {
                const T *pl = LD3Q19::ez(kb) > 0 ? bp : (LD3Q19::ez(kb) < 0 ? bm : b0);
                T r[RB::NVP];
                srec_load<T, 2 * N + 2>(pl, Sh::BPLANE, ib + LD3Q19::ex(kb) + Sh::BX * LD3Q19::ey(kb), r);
                const T eu = T(LD3Q19::ex(k)) * r[N - 1] + T(LD3Q19::ey(k)) * r[N] + T(LD3Q19::ez(k)) * r[N + 1];
                const T uu = r[2 * N + 1];
                const T sk = wk * (T(3) * eu + T(4.5) * eu * eu - T(1.5) * uu);
#pragma unroll
                for (int e = 0; e < N - 1; ++e) { acc[e] += r[e] * sk; lapS[e] += wk * (r[N + 2 + e] - r0[N + 2 + e]); }
            }
        });
        const int s0 = sxy + nxy * zc;
        bool bad = false;
#pragma unroll
        for (int e = 0; e < N - 1; ++e) {
            const T out = r0[e] + (acc[e] - cf.m * lapS[e]);   // S Laplacian as link differences (mass-exact)
            Cout[e * n + s0] = out;
            bad |= !isfinite(out);
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
        // warm-up: A-planes z_lo-2 .. z_lo+1, B-planes z_lo-1 and z_lo
        T cl[ITER][N - 1];
        T fo[19], fr[19];
#pragma unroll 1
        for (int za = z_lo - 2; za <= z_lo + 1; ++za) {
            load_A(za, cl);
            fill_A(za, cl);
        }
        __syncthreads();
        load_F(z_lo - 1, fo, fr);
        fill_B(z_lo - 1, false, fo, fr);
        load_F(z_lo, fo, fr);
        fill_B(z_lo, true, fo, fr);
        load_A(z_lo + 2, cl);
        load_F(z_lo + 1, fo, fr);
        __syncthreads();
#pragma unroll 1
        for (int zc = z_lo; zc < z_hi; ++zc) {
            fill_A(zc + 2, cl);
            __syncthreads();
            fill_B(zc + 1, zc + 1 < z_hi, fo, fr);
            __syncthreads();
            if (zc + 1 < z_hi) {               // next plane's loads fly while this plane is gathered
                load_A(zc + 3, cl);
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

template <int N, typename T, typename SF, int TX, int TY, int Q4>
cudaError_t launch_fused3d(const Geom &g, const Coef<T> &cf, const Buffers &b, int cur, cudaStream_t st) {
    using Sh = Fused3DShape<N, T, TX, TY>;
    static bool attr_done = false;
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(k_fused3d<N, T, SF, TX, TY, Q4>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(Sh::BYTES));
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    const int tiles = ((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY);
    // z-chunks: enough CTAs for about three per SM, but chunks of at least 8 planes
    int chunks = (3 * 152 + tiles - 1) / tiles;
    chunks = max(1, min(chunks, g.nz / 8));
    const int zchunk = (g.nz + chunks - 1) / chunks;
    chunks = (g.nz + zchunk - 1) / zchunk;
    const dim3 grid((g.nx + TX - 1) / TX, (g.ny + TY - 1) / TY, chunks);
    k_fused3d<N, T, SF, TX, TY, Q4><<<grid, TX * TY, Sh::BYTES, st>>>(
        g, cf, static_cast<const SF *>(b.f[cur]), static_cast<SF *>(b.f[1 - cur]),
        static_cast<const T *>(b.C[cur]), static_cast<T *>(b.C[1 - cur]), b.flag, zchunk);
    return cudaGetLastError();
}

// D3Q19 dispatch: the fused step with two tile shapes (32 x 4 and 32 x 8; the
// wider one only where its rings fit the 227 KB of shared memory of a CTA).
template <int N, typename T, typename SF>
struct Fused3DLaunch {
    static constexpr bool kWideFits = Fused3DShape<N, T, 32, 8>::BYTES <= 220 * 1024;
    static cudaError_t step(const Geom &g, const void *coef, const Buffers &b, int cur, cudaStream_t st, int variant) {
        const Coef<T> &cf = *static_cast<const Coef<T> *>(coef);
        if constexpr (kWideFits) {
            if (variant == 1) return launch_fused3d<N, T, SF, 32, 8, Q4_PARAM>(g, cf, b, cur, st);
        }
        return launch_fused3d<N, T, SF, 32, 4, Q4_PARAM>(g, cf, b, cur, st);
    }
    static const Ops *ops(int prec) {
        using B = Launch<LD3Q19, N, T, SF>;
        static const Ops o = {19, 3, N, prec, 1, {K_FUSED, K_FUSED}, {&step, nullptr}, 2,
                              {"fused3d 32x4", "fused3d 32x8", nullptr, nullptr},
                              &B::moments, &B::reduce, &B::init_f, &B::unpack_f, &B::pack_C, &B::init_g,
                              int(sizeof(SF)), int(sizeof(T))};
        return &o;
    }
};

// N = 2..4 and N = 5..8 are instantiated in separate translation units.
template <typename T, typename SF>
const Ops *ops_fused3d_lo(int N, int prec) {
    switch (N) {
        case 2: return Fused3DLaunch<2, T, SF>::ops(prec);
        case 3: return Fused3DLaunch<3, T, SF>::ops(prec);
        case 4: return Fused3DLaunch<4, T, SF>::ops(prec);
        default: return nullptr;
    }
}

template <typename T, typename SF>
const Ops *ops_fused3d_hi(int N, int prec) {
    switch (N) {
        case 5: return Fused3DLaunch<5, T, SF>::ops(prec);
        case 6: return Fused3DLaunch<6, T, SF>::ops(prec);
        case 7: return Fused3DLaunch<7, T, SF>::ops(prec);
        case 8: return Fused3DLaunch<8, T, SF>::ops(prec);
        default: return nullptr;
    }
}

}  // namespace nfe
