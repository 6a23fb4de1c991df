// Open and complex boundaries (Sec. III C; the conditions of the microfluidic and
// patterned-surface applications): the kernels besides the fused tile's geometry form (the
// outflow kernels also serve the D3Q19 split step).
//
//   k_outflow_sum / k_outflow_apply
//                   the convective outflow on the x = nx - 1 edge, after the fused step:
//                   U = mean over the fluid nodes of column nx - 2 of sum_k e_kx f_k(t+1);
//                   every population and volume fraction of a fluid node in column nx - 1
//                   becomes (old + U new(upstream)) / (1 + U); the ghost column follows
//                   with C(nx - 1, t+1).  The F/2 term of the velocity is left out (F at
//                   t+1 is not known at this point).  One thread per row (a (y, z) line;
//                   D2Q9 and D3Q19); the partial sums of U are added in a fixed order, so
//                   U is the same on every run.
//   k_inlet_table   per inlet: v_b, C_b and the flux potential S_b of the uniform state C_b
//                   (Eq. 12 without the Laplacian term), in the compute type.
//   k_geo_prepare   C := C_b on the inlet nodes; ghost := column nx - 1.
//   k_moments_geo   the FP64 fields with the node classes: a solid neighbour takes the value
//                   at x, the ghost column serves column nx - 1; solid nodes report v = P =
//                   F_s = 0, inlet nodes v = v_b, P = F_s = 0.
#pragma once

namespace nfe {

// Rows per CTA of the two outflow kernels.
constexpr int kOutflowRows = 32;

// Part 1: per CTA, the sum of sum_k e_kx f_k(t+1) over the fluid nodes of column nx - 2 in its
// rows, and their count (FP64, fixed order).  A row is one (y, z) line of the grid (rows =
// ny nz; site x + nx r), so the same kernels serve D2Q9 and D3Q19.
template <class L, typename T, typename SF>
__global__ void __launch_bounds__(kOutflowRows)
k_outflow_sum(Geom g, Coef<T> cf, const unsigned char *__restrict__ node, const SF *__restrict__ fnew,
              double *__restrict__ part, int rows) {
    __shared__ double red[kOutflowRows];
    __shared__ int cnt[kOutflowRows];
    const int nx = g.nx;
    const size_t n = size_t(g.n);
    const int tid = threadIdx.x, r = blockIdx.x * kOutflowRows + tid;
    double jx = 0.0;
    int c = 0;
    if (r < rows) {
        const size_t s = size_t(nx - 2) + size_t(nx) * r;
        if (node[s] == kNodeFluid) {
            T j = T(0);
#pragma unroll
            for (int k = 1; k < L::Q; ++k)
                if (L::ex(k) != 0) {
                    const T fk = FStore<SF, T>::load(fnew + (k - 1) * n + s, L::w(k), cf.finv);
                    j += L::ex(k) > 0 ? fk : -fk;
                }
            jx = double(j);
            c = 1;
        }
    }
    red[tid] = jx;
    cnt[tid] = c;
    __syncthreads();
    for (int o = kOutflowRows / 2; o > 0; o >>= 1) {
        if (tid < o) { red[tid] += red[tid + o]; cnt[tid] += cnt[tid + o]; }
        __syncthreads();
    }
    if (tid == 0) { part[2 * blockIdx.x] = red[0]; part[2 * blockIdx.x + 1] = double(cnt[0]); }
}

// Part 2: U from the partial sums (every CTA adds them in the same order), then the update of
// its rows of column nx - 1 and of the ghost column (ghost value e of row r at e rows + r).
template <class L, int N, typename T, typename SF>
__global__ void __launch_bounds__(kOutflowRows)
k_outflow_apply(Geom g, Coef<T> cf, const unsigned char *__restrict__ node, const SF *__restrict__ fold,
                SF *__restrict__ fnew, const T *__restrict__ Cold, T *__restrict__ Cnew,
                const T *__restrict__ gh_in, T *__restrict__ gh_out, const double *__restrict__ part, int nparts,
                int rows) {
    __shared__ double Us;
    const int nx = g.nx;
    const size_t n = size_t(g.n);
    if (threadIdx.x == 0) {
        double sum = 0.0, c = 0.0;
        for (int i = 0; i < nparts; ++i) { sum += part[2 * i]; c += part[2 * i + 1]; }
        Us = c > 0.0 ? sum / c : 0.0;
    }
    __syncthreads();
    const double U = Us;
    const T u = T(U), inv = T(1.0 / (1.0 + U));
    const int r = blockIdx.x * kOutflowRows + threadIdx.x;
    if (r >= rows) return;
    const size_t sN = size_t(nx - 1) + size_t(nx) * r, sM = size_t(nx - 2) + size_t(nx) * r;
    if (node[sN] == kNodeFluid) {
#pragma unroll
        for (int k = 1; k < L::Q; ++k) {
            const T a = FStore<SF, T>::load(fold + (k - 1) * n + sN, L::w(k), cf.finv);
            const T b = FStore<SF, T>::load(fnew + (k - 1) * n + sM, L::w(k), cf.finv);
            FStore<SF, T>::store(fnew + (k - 1) * n + sN, (a + u * b) * inv, L::w(k), cf.fscale);
        }
#pragma unroll
        for (int e = 0; e < N - 1; ++e) Cnew[e * n + sN] = (Cold[e * n + sN] + u * Cnew[e * n + sM]) * inv;
    }
#pragma unroll
    for (int e = 0; e < N - 1; ++e) gh_out[size_t(e) * rows + r] = (gh_in[size_t(e) * rows + r] + u * Cnew[e * n + sN]) * inv;
}

template <class L, int N, typename T, typename SF>
cudaError_t launch_outflow(const Geom &g, const Coef<T> &cf, const Buffers &b, int cur, cudaStream_t st) {
    const int rows = g.ny * g.nz;
    const int blocks = (rows + kOutflowRows - 1) / kOutflowRows;
    k_outflow_sum<L, T, SF><<<blocks, kOutflowRows, 0, st>>>(g, cf, b.node, static_cast<const SF *>(b.f[1 - cur]), b.opart,
                                                             rows);
    k_outflow_apply<L, N, T, SF><<<blocks, kOutflowRows, 0, st>>>(
        g, cf, b.node, static_cast<const SF *>(b.f[cur]), static_cast<SF *>(b.f[1 - cur]),
        static_cast<const T *>(b.C[cur]), static_cast<T *>(b.C[1 - cur]),
        static_cast<const T *>(b.ghost[cur]), static_cast<T *>(b.ghost[1 - cur]), b.opart, blocks, rows);
    return cudaGetLastError();
}

template <int N, typename T, typename SF>
cudaError_t launch_outflow2d(const Geom &g, const Coef<T> &cf, const Buffers &b, int cur, cudaStream_t st) {
    return launch_outflow<LD2Q9, N, T, SF>(g, cf, b, cur, st);
}

// rows: K x (2 + N) FP64 (vx, vy, C_b in internal order); out: K x 2N in the compute type.
template <int N, typename T>
__global__ void k_inlet_table(Coef<T> cf, const double *__restrict__ rows, int K, T *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= K) return;
    const double *r = rows + size_t(j) * (2 + N);
    T c[N];
#pragma unroll
    for (int a = 0; a < N; ++a) c[a] = T(r[2 + a]);
    T q[N - 1], S[N - 1];
    flux_poly<N, T, Q4_GLOBAL>(c, cf, q);
#pragma unroll
    for (int e = 0; e < N - 1; ++e) S[e] = c[e] * q[e];
    flux_rest<N, T, Q4_GLOBAL>(c, cf, S);
    T *o = out + size_t(j) * (2 * N);
    o[0] = T(r[0]);
    o[1] = T(r[1]);
#pragma unroll
    for (int e = 0; e < N - 1; ++e) { o[2 + e] = c[e]; o[N + 1 + e] = S[e]; }
}

template <int N, typename T>
__global__ void k_geo_prepare(Geom g, const unsigned char *__restrict__ node, const T *__restrict__ inl,
                              T *__restrict__ C, T *__restrict__ ghost, int outflow) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const size_t n = size_t(g.n);
    if (s < g.n) {
        const unsigned char cls = node[s];
        if (cls >= kNodeInlet0) {
            const T *row = inl + (cls - kNodeInlet0) * (2 * N);
#pragma unroll
            for (int e = 0; e < N - 1; ++e) C[e * n + s] = row[2 + e];
        }
    }
    // column nx - 1 holds no inlet node, so these reads do not race with the writes above
    if (outflow && s < g.ny) {
#pragma unroll
        for (int e = 0; e < N - 1; ++e) ghost[e * g.ny + s] = C[e * n + (g.nx - 1) + size_t(g.nx) * s];
    }
}

template <int N, typename T, typename SF>
__global__ void k_moments_geo(Geom g, Coef<T> cf, const SF *__restrict__ fin, const T *__restrict__ C,
                              const unsigned char *__restrict__ node, const T *__restrict__ inl,
                              const T *__restrict__ ghost, int outflow, double *__restrict__ out,
                              int *__restrict__ flag) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.n) return;
    const int nx = g.nx, ny = g.ny;
    const int x = s % nx, y = s / nx;
    const size_t n = size_t(g.n);
    Stencil<LD2Q9, N, T> st;
    T rest = T(0);
#pragma unroll
    for (int a = 0; a < N - 1; ++a) { st.c[a] = C[a * n + s]; rest += st.c[a]; }
    st.c[N - 1] = T(1) - rest;
    const unsigned char cls = node[s];
    T v0 = T(0), v1 = T(0), P = T(0), Fs[3] = {T(0), T(0), T(0)};
    bool bad = false;
    if (cls == kNodeFluid) {
        const T E0 = bulk_energy<N, T>(st.c, cf);
#pragma unroll
        for (int a = 0; a < N; ++a) { st.lap[a] = T(0); st.gr[a][0] = st.gr[a][1] = st.gr[a][2] = T(0); }
        st.gE[0] = st.gE[1] = st.gE[2] = T(0);
#pragma unroll
        for (int k = 1; k < 9; ++k) {
            const int xx = x + LD2Q9::ex(k), yy = y + LD2Q9::ey(k);
            if ((g.wx && (xx < 0 || xx >= nx)) || (g.wy && (yy < 0 || yy >= ny))) continue;   // mirror rule
            const int yw = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
            const bool gcol = outflow && xx == nx;
            const int xw = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
            const int j = (gcol ? nx - 1 : xw) + nx * yw;
            if (node[j] == kNodeSolid) continue;                                                  // mirror rule
            T cn[N];
            T r2 = T(0);
#pragma unroll
            for (int a = 0; a < N - 1; ++a) { cn[a] = gcol ? ghost[a * ny + yw] : C[a * n + j]; r2 += cn[a]; }
            cn[N - 1] = T(1) - r2;
            const T wk = T(LD2Q9::w(k));
#pragma unroll
            for (int a = 0; a < N; ++a) {
                const T d = cn[a] - st.c[a];
                st.lap[a] += wk * d;
                if (LD2Q9::ex(k)) st.gr[a][0] += (LD2Q9::ex(k) > 0 ? wk : -wk) * d;
                if (LD2Q9::ey(k)) st.gr[a][1] += (LD2Q9::ey(k) > 0 ? wk : -wk) * d;
            }
            const T dE = bulk_energy<N, T>(cn, cf) - E0;
            if (LD2Q9::ex(k)) st.gE[0] += (LD2Q9::ex(k) > 0 ? wk : -wk) * dE;
            if (LD2Q9::ey(k)) st.gE[1] += (LD2Q9::ey(k) > 0 ? wk : -wk) * dE;
        }
#pragma unroll
        for (int a = 0; a < N; ++a) { st.lap[a] *= T(6); st.gr[a][0] *= T(3); st.gr[a][1] *= T(3); }
        st.gE[0] *= T(3); st.gE[1] *= T(3);
        T S[N - 1];
        force_and_potential<LD2Q9, N, T>(cf, st, Fs, S);
        T sumf = T(0), j0 = T(0), j1 = T(0);
#pragma unroll
        for (int k = 1; k < 9; ++k) {
            const T fk = FStore<SF, T>::load(fin + (k - 1) * n + s, LD2Q9::w(k), cf.finv);
            bad |= !isfinite(fk);
            sumf += fk;
            if (LD2Q9::ex(k)) j0 += LD2Q9::ex(k) > 0 ? fk : -fk;
            if (LD2Q9::ey(k)) j1 += LD2Q9::ey(k) > 0 ? fk : -fk;
        }
        T cc = T(0);                      // body force on one component, F += C_c F_c
#pragma unroll
        for (int a = 0; a < N; ++a) cc += cf.fcsel[a] * st.c[a];
        v0 = j0 + T(0.5) * (Fs[0] + cf.fb[0] + cc * cf.fc[0]);
        v1 = j1 + T(0.5) * (Fs[1] + cf.fb[1] + cc * cf.fc[1]);
        const T w0 = T(LD2Q9::w(0));
        P = (sumf - T(1.5) * w0 * (v0 * v0 + v1 * v1)) * T(1.0 / (3.0 * (1.0 - LD2Q9::w(0))));
    } else if (cls != kNodeSolid) {
        const T *row = inl + (cls - kNodeInlet0) * (2 * N);
        v0 = row[0];
        v1 = row[1];
    }
#pragma unroll
    for (int a = 0; a < N; ++a) {
        out[size_t(cf.uidx[a]) * n + s] = double(st.c[a]);
        bad |= !isfinite(st.c[a]);
    }
    out[(N + 0) * n + s] = double(v0);
    out[(N + 1) * n + s] = double(v1);
    out[(N + 2) * n + s] = 0.0;
    out[(N + 3) * n + s] = double(P);
    out[(N + 4) * n + s] = double(Fs[0]);
    out[(N + 5) * n + s] = double(Fs[1]);
    out[(N + 6) * n + s] = 0.0;
    if (bad) atomicOr(flag, 1);
}

template <int N, typename T, typename SF>
struct GeoOps {
    static cudaError_t inlet_table(const void *coef, const double *rows, int K, void *out, cudaStream_t st) {
        const Coef<T> &cf = *static_cast<const Coef<T> *>(coef);
        k_inlet_table<N, T><<<1, kMaxInlets, 0, st>>>(cf, rows, K, static_cast<T *>(out));
        return cudaGetLastError();
    }
    static cudaError_t prepare(const Geom &g, const Buffers &b, int cur, int, cudaStream_t st) {
        k_geo_prepare<N, T><<<blocks_for(g.n, 256), 256, 0, st>>>(g, b.node, static_cast<const T *>(b.inl),
                                                                  static_cast<T *>(b.C[cur]),
                                                                  static_cast<T *>(b.ghost[cur]), b.outflow);
        return cudaGetLastError();
    }
    static cudaError_t moments(const Geom &g, const void *coef, const Buffers &b, int cur, cudaStream_t st) {
        const Coef<T> &cf = *static_cast<const Coef<T> *>(coef);
        k_moments_geo<N, T, SF><<<blocks_for(g.n, 256), 256, 0, st>>>(
            g, cf, static_cast<const SF *>(b.f[cur]), static_cast<const T *>(b.C[cur]), b.node,
            static_cast<const T *>(b.inl), static_cast<const T *>(b.ghost[cur]), b.outflow, b.fields, b.flag);
        return cudaGetLastError();
    }
};

}  // namespace nfe
