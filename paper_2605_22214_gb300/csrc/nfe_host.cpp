// Host side of the C ABI declared in include/nfe.h: validation, the Sec. II
// tables, device memory, CUDA-graph replay of the time step, checkpoints,
// diagnostics and kernel timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <map>
#include <utility>

#include "nfe_batch.h"
#include "nfe_internal.h"
#include "nfe_spectrum.h"
#include "nfe_tables.h"

using namespace nfe;

namespace {

thread_local std::string g_err;

nfe_status fail(nfe_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

nfe_status cuda_fail(cudaError_t e, const char *what) {
    cudaGetLastError();   // a non-sticky error is reported here once, not again by the next call
    return fail(NFE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                                    \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);         \
    } while (0)

const Ops *select_ops(int lattice, int N, int prec) {
    if (lattice == NFE_D2Q9) {
        switch (prec) {
            case NFE_FP64: return ops_d2q9_fp64(N);
            case NFE_FP32: return ops_d2q9_fp32(N);
            case NFE_FP32_F16STORE: return ops_d2q9_f16(N);
            case NFE_FP32_BF16STORE: return ops_d2q9_bf16(N);
        }
    } else if (lattice == NFE_D3Q19) {
        switch (prec) {
            case NFE_FP64: return ops_d3q19_fp64(N);
            case NFE_FP32: return ops_d3q19_fp32(N);
            case NFE_FP32_F16STORE: return ops_d3q19_f16(N);
            case NFE_FP32_BF16STORE: return ops_d3q19_bf16(N);
        }
    }
    return nullptr;
}

}  // namespace

nfe_status nfe::set_error(nfe_status s, const char *msg) {
    g_err = msg ? msg : "";
    return s;
}

namespace {

struct TimedLaunch {
    int kind;
    cudaEvent_t a, b;
};

}  // namespace

struct nfe_sim {
    nfe_grid grid{};
    int N = 0;
    int prec = 0;
    Geom geom{};
    const Ops *ops = nullptr;
    Tables tab;
    Coef<double> cd{};
    Coef<float> cfl{};
    const void *coef = nullptr;       // points at cd or cfl
    void *q4dev = nullptr;
    void *r3dev = nullptr;            // no-phi remainder table
    Spectrum *spectrum = nullptr;     // domain-size diagnostic (cuFFT plan + scratch), on first use
    Buffers buf{};
    int uidx[NFE_MAX_N] = {0};        // internal slot -> user component
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int64_t step = 0;
    size_t fplanes_bytes = 0, cplanes_bytes = 0, gplanes_bytes = 0;   // gplanes: stored g (tau_g != 1)
    double tau_g = 1.0;
    bool no_phi = false;
    // D2Q9 geometry (nfe_set_geometry): device node classes, inlet table and ghost column
    unsigned char *node_dev = nullptr;
    void *inl_dev = nullptr;
    int ninlets = 0;
    size_t ghost_bytes = 0;           // one ghost buffer ((N-1) x ny nz), 0 without an outflow
    size_t geo_bytes = 0;             // device bytes held by the geometry
    nfe_alloc_fn ualloc = nullptr;    // caller's device allocator (null: cudaMalloc)
    nfe_free_fn ufree = nullptr;
    void *uctx = nullptr;
    size_t fields_planes = 0;
    size_t device_bytes = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    int variant = -1;                 // tile shape; -1 until the autotuner has run
    bool profiling = false;
    std::vector<TimedLaunch> timed;
    std::vector<cudaEvent_t> event_pool;
    int64_t prof_launches[K_NKINDS] = {0};
    double prof_ms[K_NKINDS] = {0};
};

namespace {

template <typename T>
void fill_coef(const nfe_sim &s, const nfe_params &p, Coef<T> &c) {
    const int N = s.N;
    std::memset(&c, 0, sizeof c);
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) {
            c.beta[a][b] = T(s.tab.beta[a * N + b]);
            c.kappa[a][b] = T(s.tab.kappa[a * N + b]);
        }
    const int m2 = N * (N + 1) / 2;
    for (int e = 0; e < N - 1; ++e)
        for (int j = 0; j < m2; ++j) c.q2[e][j] = T(s.tab.q2[e * m2 + j]);
    for (int a = 0; a < N; ++a) {
        const double tau = p.tau[s.uidx[a]];
        c.omp[a] = T(1.0 / tau);
        c.omm[a] = p.lambda_trt < 0.0 ? T(1.0 / tau) : T(1.0 / (p.lambda_trt / (tau - 0.5) + 0.5));
        c.uidx[a] = s.uidx[a];
    }
    c.uniform_tau = 1;
    for (int a = 1; a < N; ++a)
        if (c.omp[a] != c.omp[0] || c.omm[a] != c.omm[0]) c.uniform_tau = 0;
    c.m = T(p.m);
    c.d34 = T(0.75 * p.D);
    for (int d = 0; d < 3; ++d) c.fb[d] = T(p.body_force[d]);
    c.has_fc = (p.component_force[0] != 0.0 || p.component_force[1] != 0.0 || p.component_force[2] != 0.0) ? 1 : 0;
    for (int d = 0; d < 3; ++d) c.fc[d] = T(p.component_force[d]);
    for (int a = 0; a < N; ++a) c.fcsel[a] = T(c.has_fc && s.uidx[a] == p.component_force_index ? 1 : 0);
    const double sc = (s.prec == NFE_FP32_F16STORE) ? std::ldexp(1.0, p.scale_exp) : 1.0;
    c.fscale = T(sc);
    c.finv = T(1.0 / sc);
    c.has_q4 = s.tab.omega != 0.0 ? 1 : 0;
    c.nonconservative = (p.flags & NFE_NONCONSERVATIVE_FORCE) ? 1 : 0;
    c.q4 = static_cast<const T *>(s.q4dev);
    c.r3 = static_cast<const T *>(s.r3dev);
    c.no_phi = (p.flags & NFE_NO_PHI) ? 1 : 0;
    c.gomega = T(1.0 / s.tau_g);
    if (N <= kQ4InlineMaxN)
        for (size_t j = 0; j < s.tab.q4.size(); ++j) c.q4c[j] = T(s.tab.q4[j]);
}

void dev_free(nfe_sim *s, void *p) {
    if (!p) return;
    if (s->ufree) s->ufree(p, s->uctx);
    else cudaFree(p);
}

nfe_status free_all(nfe_sim *s) {
    for (auto &g : s->graph) if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    for (auto &t : s->timed) { s->event_pool.push_back(t.a); s->event_pool.push_back(t.b); }
    s->timed.clear();
    for (auto e : s->event_pool) cudaEventDestroy(e);
    s->event_pool.clear();
    void *ptrs[] = {s->buf.f[0], s->buf.f[1], s->buf.C[0], s->buf.C[1],
                    s->buf.fields, s->buf.partials, s->buf.diag, s->buf.flag, s->q4dev, s->r3dev,
                    s->buf.g[0], s->buf.g[1], s->node_dev, s->inl_dev, s->buf.ghost[0], s->buf.ghost[1],
                    s->buf.opart, s->buf.lmask, s->buf.vs};
    for (void *p : ptrs) dev_free(s, p);
    std::memset(&s->buf, 0, sizeof s->buf);
    s->q4dev = nullptr;
    s->r3dev = nullptr;
    s->node_dev = nullptr;
    s->inl_dev = nullptr;
    spectrum_destroy(s->spectrum);
    s->spectrum = nullptr;
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    s->stream = nullptr;
    return NFE_OK;
}

nfe_status dev_alloc(nfe_sim *s, void **p, size_t bytes) {
    if (s->ualloc) {
        *p = s->ualloc(bytes, s->uctx);
        if (!*p) return fail(NFE_ENOMEM, "device_alloc returned NULL for %zu bytes", bytes);
        if (reinterpret_cast<uintptr_t>(*p) % 256 != 0) {
            s->ufree(*p, s->uctx);
            *p = nullptr;
            return fail(NFE_ENOMEM, "device_alloc returned memory not aligned to 256 bytes");
        }
        s->device_bytes += bytes;
        return NFE_OK;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(NFE_ENOMEM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    s->device_bytes += bytes;
    return NFE_OK;
}

cudaEvent_t get_event(nfe_sim *s) {
    if (!s->event_pool.empty()) {
        cudaEvent_t e = s->event_pool.back();
        s->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// one time step from buffer `cur`, optionally with events around each kernel
// The variant a step really runs: the D3Q19 no-phi ablation and stored component populations
// (tau_g != 1) exist in the split form only, so its fused variants (0: 32x4, 1: 32x8) run the split
// form with the same physics tile.
int effective_variant(const nfe_sim *s, int variant) {
    const int v = variant < 0 ? 0 : variant;
    if (s->buf.node && s->ops->Q == 19) return 3;      // the D3Q19 geometry kernels: one split form
    if ((s->no_phi || s->buf.g[0]) && s->ops->Q == 19 && v < 2) return v == 0 ? 3 : 2;
    return v;
}

nfe_status launch_step(nfe_sim *s, int cur, bool timed, int variant) {
    const int v = effective_variant(s, variant);
    variant = v;
    const bool own_list = s->ops->vnk[v] > 0;            // a variant with its own kernel list
    const int nk = own_list ? s->ops->vnk[v] : s->ops->nk;
    const int *kinds = own_list ? s->ops->vkinds[v] : s->ops->kinds;
    for (int i = 0; i < nk; ++i) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (timed) { a = get_event(s); b = get_event(s); CK(cudaEventRecord(a, s->stream)); }
        CK(s->ops->kern[i](s->geom, s->coef, s->buf, cur, s->stream, variant));
        if (timed) {
            CK(cudaEventRecord(b, s->stream));
            s->timed.push_back({kinds[i], a, b});
        }
    }
    return NFE_OK;
}

// Pick the fastest tile shape by timing each variant on the current state.  A
// step reads buffer cur and writes buffer 1 - cur, so the state is untouched.
nfe_status autotune(nfe_sim *s) {
    if (s->variant >= 0) return NFE_OK;
    // the geometry form has one tile shape whatever the variant
    if (s->ops->nvariants <= 1 || s->buf.node) { s->variant = 0; return NFE_OK; }
    cudaEvent_t a = get_event(s), b = get_event(s);
    double best = 1e300;
    int best_v = 0;
    const int reps = s->geom.n > (1 << 22) ? 3 : 10;
    for (int v = 0; v < s->ops->nvariants; ++v) {
        nfe_status st;
        for (int r = 0; r < 2; ++r)
            if ((st = launch_step(s, s->buf.cur, false, v)) != NFE_OK) return st;
        CK(cudaEventRecord(a, s->stream));
        for (int r = 0; r < reps; ++r)
            if ((st = launch_step(s, s->buf.cur, false, v)) != NFE_OK) return st;
        CK(cudaEventRecord(b, s->stream));
        CK(cudaEventSynchronize(b));
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, a, b));
        if (ms < best) { best = ms; best_v = v; }
    }
    s->event_pool.push_back(a);
    s->event_pool.push_back(b);
    CK(cudaMemsetAsync(s->buf.flag, 0, sizeof(int), s->stream));
    s->variant = best_v;
    return NFE_OK;
}

nfe_status ensure_graph(nfe_sim *s, int cur) {
    if (s->graph[cur]) return NFE_OK;
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    nfe_status st = launch_step(s, cur, false, s->variant);
    if (st == NFE_OK) st = launch_step(s, 1 - cur, false, s->variant);
    cudaError_t e = cudaStreamEndCapture(s->stream, &g);
    if (st != NFE_OK) { if (g) cudaGraphDestroy(g); cudaGetLastError(); return st; }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&s->graph[cur], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { s->graph[cur] = nullptr; return cuda_fail(e, "cudaGraphInstantiate"); }
    return NFE_OK;
}

nfe_status ensure_fields(nfe_sim *s) {
    if (s->buf.fields) return NFE_OK;
    nfe_status st = dev_alloc(s, reinterpret_cast<void **>(&s->buf.fields),
                              s->fields_planes * size_t(s->geom.n) * sizeof(double));
    if (st != NFE_OK) return st;
    st = dev_alloc(s, reinterpret_cast<void **>(&s->buf.partials),
                   size_t(kReduceBlocks) * diag_count(s->N) * sizeof(double));
    if (st != NFE_OK) return st;
    return dev_alloc(s, reinterpret_cast<void **>(&s->buf.diag), diag_count(s->N) * sizeof(double));
}

// fields of the current state (FP64 planes in bufs.fields), with the node classes when the
// grid has a geometry
cudaError_t run_moments(nfe_sim *s) {
    if (s->buf.node) return s->ops->moments_geo(s->geom, s->coef, s->buf, s->buf.cur, s->stream);
    return s->ops->moments(s->geom, s->coef, s->buf, s->buf.cur, s->stream);
}

size_t state_size(const nfe_sim *s) {
    return sizeof(int64_t) + s->fplanes_bytes + s->cplanes_bytes + s->gplanes_bytes + s->ghost_bytes;
}

void geo_free(nfe_sim *s) {
    void *ptrs[] = {s->node_dev, s->inl_dev, s->buf.ghost[0], s->buf.ghost[1], s->buf.opart, s->buf.lmask};
    for (void *p : ptrs) dev_free(s, p);
    s->buf.opart = nullptr;
    s->buf.lmask = nullptr;
    s->device_bytes -= s->geo_bytes;
    s->geo_bytes = 0;
    s->node_dev = nullptr;
    s->inl_dev = nullptr;
    s->buf.node = nullptr;
    s->buf.inl = nullptr;
    s->buf.ghost[0] = s->buf.ghost[1] = nullptr;
    s->buf.outflow = 0;
    s->ninlets = 0;
    s->ghost_bytes = 0;
}

nfe_status check_sim(const nfe_sim *s) {
    if (!s) return fail(NFE_EINVAL, "sim is NULL");
    return NFE_OK;
}

}  // namespace

extern "C" {

const char *nfe_status_string(nfe_status s) {
    switch (s) {
        case NFE_OK: return "ok";
        case NFE_EINVAL: return "invalid argument";
        case NFE_ENOMEM: return "out of memory";
        case NFE_ECUDA: return "CUDA error";
        case NFE_ESINGULAR: return "singular alpha/Lambda/Theta system";
        case NFE_ENONFINITE: return "non-finite volume fraction";
        case NFE_ETIMEOUT: return "device wait timed out";
        case NFE_EUNSUPPORTED: return "unsupported combination";
    }
    return "unknown status";
}

const char *nfe_last_error(void) { return g_err.c_str(); }

nfe_status nfe_create(const nfe_grid *grid, int N, const nfe_params *p, nfe_sim **out) {
    if (!out) return fail(NFE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!grid || !p) return fail(NFE_EINVAL, "grid or params is NULL");
    if (grid->lattice != NFE_D2Q9 && grid->lattice != NFE_D3Q19) return fail(NFE_EINVAL, "lattice must be NFE_D2Q9 or NFE_D3Q19");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return fail(NFE_EINVAL, "grid sizes must be >= 1");
    if (grid->lattice == NFE_D2Q9 && (grid->nz != 1 || (grid->wall_mask & NFE_WALL_Z)))
        return fail(NFE_EINVAL, "D2Q9 needs nz = 1 and no z walls");
    if (grid->wall_mask & ~7u) return fail(NFE_EINVAL, "unknown wall bits");
    const long long n = (long long)grid->nx * grid->ny * grid->nz;
    if (n > (1LL << 31) - 4096) return fail(NFE_EINVAL, "grid has %lld sites; the limit is 2^31 - 4096", n);
    if (N < 2 || N > NFE_MAX_N) return fail(NFE_EINVAL, "N = %d outside 2..%d", N, NFE_MAX_N);
    if (!p->sigma || !p->tau) return fail(NFE_EINVAL, "sigma or tau is NULL");
    double smax = 0.0;
    for (int i = 0; i < N * N; ++i) smax = std::fmax(smax, std::fabs(p->sigma[i]));
    for (int i = 0; i < N; ++i) {
        if (p->sigma[i * N + i] != 0.0) return fail(NFE_EINVAL, "sigma[%d][%d] must be 0", i, i);
        for (int j = 0; j < N; ++j) {
            if (i == j) continue;
            if (!(p->sigma[i * N + j] > 0.0) || !std::isfinite(p->sigma[i * N + j]))
                return fail(NFE_EINVAL, "sigma[%d][%d] must be positive and finite", i, j);
            if (std::fabs(p->sigma[i * N + j] - p->sigma[j * N + i]) > 1e-15 * smax)
                return fail(NFE_EINVAL, "sigma is not symmetric at (%d, %d)", i, j);
        }
        if (!(p->tau[i] > 0.5) || !std::isfinite(p->tau[i])) return fail(NFE_EINVAL, "tau[%d] must be > 1/2", i);
    }
    if (!(p->D > 0.0) || !std::isfinite(p->D)) return fail(NFE_EINVAL, "D must be positive");
    if (!(p->m >= 0.0) || !std::isfinite(p->m)) return fail(NFE_EINVAL, "m must be >= 0");
    if (!std::isfinite(p->lambda_trt)) return fail(NFE_EINVAL, "lambda_trt must be finite");
    if (!std::isnan(p->omega_stab) && !(p->omega_stab >= 0.0)) return fail(NFE_EINVAL, "omega_stab must be >= 0 or NaN");
    for (int d = 0; d < 3; ++d) if (!std::isfinite(p->body_force[d])) return fail(NFE_EINVAL, "body force must be finite");
    for (int d = 0; d < 3; ++d) if (!std::isfinite(p->component_force[d])) return fail(NFE_EINVAL, "component force must be finite");
    if ((p->component_force[0] != 0.0 || p->component_force[1] != 0.0 || p->component_force[2] != 0.0) &&
        (p->component_force_index < 0 || p->component_force_index >= N))
        return fail(NFE_EINVAL, "component_force_index out of range");
    if (p->implicit_component < 0 || p->implicit_component >= N) return fail(NFE_EINVAL, "implicit_component out of range");
    if (p->precision < NFE_FP64 || p->precision > NFE_FP32_BF16STORE) return fail(NFE_EINVAL, "unknown precision");
    if (p->flags & ~(NFE_NONCONSERVATIVE_FORCE | NFE_NO_PHI)) return fail(NFE_EINVAL, "unknown flags");
    const double tau_g = p->tau_g == 0.0 ? 1.0 : p->tau_g;
    if (!(tau_g > 0.5) || !std::isfinite(tau_g)) return fail(NFE_EINVAL, "tau_g must be > 1/2 (0 selects 1)");
    const bool stored_g = tau_g != 1.0;
    if (stored_g && (p->flags & NFE_NO_PHI)) return fail(NFE_EUNSUPPORTED, "tau_g != 1 together with NFE_NO_PHI");
    if (p->precision == NFE_FP32_F16STORE && (p->scale_exp < -20 || p->scale_exp > 20))
        return fail(NFE_EINVAL, "scale_exp outside -20..20");

    if ((p->device_alloc == nullptr) != (p->device_free == nullptr))
        return fail(NFE_EINVAL, "set both device_alloc and device_free, or neither");
    nfe_sim *s = new (std::nothrow) nfe_sim();
    if (!s) return fail(NFE_ENOMEM, "host allocation failed");
    s->ualloc = p->device_alloc;
    s->ufree = p->device_free;
    s->uctx = p->alloc_ctx;
    s->grid = *grid;
    s->N = N;
    s->prec = p->precision;
    s->geom = Geom{grid->nx, grid->ny, grid->nz, (grid->wall_mask & NFE_WALL_X) ? 1 : 0,
                   (grid->wall_mask & NFE_WALL_Y) ? 1 : 0, (grid->wall_mask & NFE_WALL_Z) ? 1 : 0, n};
    int a = 0;
    for (int c = 0; c < N; ++c) if (c != p->implicit_component) s->uidx[a++] = c;
    s->uidx[N - 1] = p->implicit_component;

    const double omega = std::isnan(p->omega_stab) ? (auto_omega(N, p->sigma) ? 1.0 / 90.0 : 0.0) : p->omega_stab;
    std::string err;
    nfe_status st = build_tables(N, p->sigma, s->uidx, p->D, omega, !(p->flags & NFE_NO_PHI), s->tab, err);
    if (st != NFE_OK) { delete s; return fail(st, "%s", err.c_str()); }
    s->ops = select_ops(grid->lattice, N, p->precision);
    if (!s->ops) { delete s; return fail(NFE_EUNSUPPORTED, "no kernels for this lattice/N/precision"); }

    if (p->cuda_stream) {
        s->stream = static_cast<cudaStream_t>(p->cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreate(&s->stream);
        if (e != cudaSuccess) { delete s; return cuda_fail(e, "cudaStreamCreate"); }
        s->own_stream = true;
    }
    const int Q = s->ops->Q;
    s->fplanes_bytes = size_t(Q - 1) * n * s->ops->f_elem_bytes;
    s->cplanes_bytes = size_t(N - 1) * n * s->ops->c_elem_bytes;
    s->gplanes_bytes = stored_g ? size_t(N - 1) * Q * n * s->ops->c_elem_bytes : 0;
    s->tau_g = tau_g;
    s->no_phi = (p->flags & NFE_NO_PHI) != 0;
    s->fields_planes = size_t(std::max(N + 7, Q - 1));
    const size_t ce = s->ops->c_elem_bytes;
#define ALLOC(ptr, bytes) do { st = dev_alloc(s, reinterpret_cast<void **>(&(ptr)), (bytes)); \
        if (st != NFE_OK) { free_all(s); delete s; return st; } } while (0)
    ALLOC(s->buf.f[0], s->fplanes_bytes);
    ALLOC(s->buf.f[1], s->fplanes_bytes);
    ALLOC(s->buf.C[0], s->cplanes_bytes);
    ALLOC(s->buf.C[1], s->cplanes_bytes);
    ALLOC(s->buf.flag, sizeof(int));
    if (stored_g) {
        ALLOC(s->buf.g[0], s->gplanes_bytes);
        ALLOC(s->buf.g[1], s->gplanes_bytes);
    }
    if (s->ops->scratch_planes > 0) ALLOC(s->buf.vs, size_t(s->ops->scratch_planes) * n * ce);
    if (!s->tab.q4.empty()) ALLOC(s->q4dev, s->tab.q4.size() * ce);
    if (!s->tab.r3.empty()) ALLOC(s->r3dev, s->tab.r3.size() * ce);
#undef ALLOC
    // upload the quartic and no-phi tables in the arithmetic type
    const std::pair<void *, const std::vector<double> *> uploads[] = {{s->q4dev, &s->tab.q4}, {s->r3dev, &s->tab.r3}};
    for (const auto &u : uploads) {
        if (!u.first) continue;
        cudaError_t e;
        if (s->prec == NFE_FP64) {
            e = cudaMemcpy(u.first, u.second->data(), u.second->size() * sizeof(double), cudaMemcpyHostToDevice);
        } else {
            std::vector<float> tmp(u.second->begin(), u.second->end());
            e = cudaMemcpy(u.first, tmp.data(), tmp.size() * sizeof(float), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) { free_all(s); delete s; return cuda_fail(e, "upload coefficient tables"); }
    }
    if (s->prec == NFE_FP64) { fill_coef<double>(*s, *p, s->cd); s->coef = &s->cd; }
    else { fill_coef<float>(*s, *p, s->cfl); s->coef = &s->cfl; }

    cudaError_t e = cudaMemsetAsync(s->buf.f[0], 0, s->fplanes_bytes, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->buf.C[0], 0, s->cplanes_bytes, s->stream);
    if (e == cudaSuccess && s->buf.g[0]) e = cudaMemsetAsync(s->buf.g[0], 0, s->gplanes_bytes, s->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->buf.flag, 0, sizeof(int), s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) { free_all(s); delete s; return cuda_fail(e, "initialise state"); }
    s->buf.cur = 0;
    *out = s;
    return NFE_OK;
}

void nfe_destroy(nfe_sim *s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    free_all(s);
    delete s;
}

nfe_status nfe_set_fields(nfe_sim *s, const double *C, const double *v) {
    nfe_status st = check_sim(s);
    if (st != NFE_OK) return st;
    if (!C) return fail(NFE_EINVAL, "C is NULL");
    if ((st = ensure_fields(s)) != NFE_OK) return st;
    const size_t n = size_t(s->geom.n);
    const int N = s->N;
    // evolved components in internal order, FP64, into the fields scratch
    for (int e = 0; e < N - 1; ++e)
        CK(cudaMemcpyAsync(s->buf.fields + e * n, C + size_t(s->uidx[e]) * n, n * sizeof(double),
                           cudaMemcpyHostToDevice, s->stream));
    CK(s->ops->pack_C(s->geom, s->buf, 0, s->buf.fields, s->stream));
    if (v) {
        CK(cudaMemcpyAsync(s->buf.fields + (N - 1) * n, v, 3 * n * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        CK(s->ops->init_f(s->geom, s->coef, s->buf, 0, s->buf.fields + (N - 1) * n, s->stream));
    } else {
        CK(cudaMemsetAsync(s->buf.f[0], 0, s->fplanes_bytes, s->stream));
    }
    // stored g (tau_g != 1): g = g^eq(C, v, S(C)) at the start
    if (s->buf.g[0]) CK(s->ops->init_g(s->geom, s->coef, s->buf, 0, v ? s->buf.fields + (N - 1) * n : nullptr, s->stream));
    // geometry: C := C_b on the inlet nodes, ghost column := column nx - 1
    if (s->buf.node) CK(s->ops->geo_prepare(s->geom, s->buf, 0, s->ninlets, s->stream));
    CK(cudaMemsetAsync(s->buf.flag, 0, sizeof(int), s->stream));
    CK(cudaStreamSynchronize(s->stream));
    s->buf.cur = 0;
    s->step = 0;
    return NFE_OK;
}

nfe_status nfe_step(nfe_sim *s, int64_t nsteps) {
    nfe_status st = check_sim(s);
    if (st != NFE_OK) return st;
    if (nsteps < 0) return fail(NFE_EINVAL, "nsteps < 0");
    if (nsteps > 0 && (st = autotune(s)) != NFE_OK) return st;
    if (s->profiling) {
        for (int64_t i = 0; i < nsteps; ++i) {
            if ((st = launch_step(s, s->buf.cur, true, s->variant)) != NFE_OK) return st;
            s->buf.cur ^= 1;
            s->step++;
        }
        return NFE_OK;
    }
    while (nsteps >= 2) {
        if ((st = ensure_graph(s, s->buf.cur)) != NFE_OK) return st;
        CK(cudaGraphLaunch(s->graph[s->buf.cur], s->stream));
        nsteps -= 2;
        s->step += 2;
    }
    if (nsteps == 1) {
        if ((st = launch_step(s, s->buf.cur, false, s->variant)) != NFE_OK) return st;
        s->buf.cur ^= 1;
        s->step++;
    }
    return NFE_OK;
}

nfe_status nfe_sync(nfe_sim *s) {
    nfe_status st = check_sim(s);
    if (st != NFE_OK) return st;
    CK(cudaStreamSynchronize(s->stream));
    int flag = 0;
    CK(cudaMemcpy(&flag, s->buf.flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) return fail(NFE_ENONFINITE, "a volume fraction became NaN or Inf");
    return NFE_OK;
}

nfe_status nfe_fields(nfe_sim *s, double *C, double *v, double *P) {
    nfe_status st = check_sim(s);
    if (st != NFE_OK) return st;
    if ((st = ensure_fields(s)) != NFE_OK) return st;
    CK(run_moments(s));
    const size_t n = size_t(s->geom.n);
    const int N = s->N;
    if (C) CK(cudaMemcpyAsync(C, s->buf.fields, N * n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    if (v) CK(cudaMemcpyAsync(v, s->buf.fields + N * n, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    if (P) CK(cudaMemcpyAsync(P, s->buf.fields + (N + 3) * n, n * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return NFE_OK;
}

nfe_status nfe_populations(nfe_sim *s, double *f) {
    nfe_status st = check_sim(s);
    if (st != NFE_OK) return st;
    if (!f) return fail(NFE_EINVAL, "f is NULL");
    if ((st = ensure_fields(s)) != NFE_OK) return st;
    CK(s->ops->unpack_f(s->geom, s->coef, s->buf, s->buf.cur, s->buf.fields, s->stream));
    CK(cudaMemcpyAsync(f, s->buf.fields, size_t(s->ops->Q - 1) * s->geom.n * sizeof(double),
                       cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return NFE_OK;
}

nfe_status nfe_domain_size(nfe_sim *s, double *L, int component, int nbins, double *Sk) {
    nfe_status st = check_sim(s);
    if (st != NFE_OK) return st;
    if (!L) return fail(NFE_EINVAL, "L is NULL");
    if (nbins < 0 || nbins > (1 << 20)) return fail(NFE_EINVAL, "nbins must be 0..2^20");
    if (nbins > 0 && (!Sk || component < 0 || component >= s->N))
        return fail(NFE_EINVAL, "S(k) wanted: Sk must be non-NULL and component in 0..N-1");
    if ((st = ensure_fields(s)) != NFE_OK) return st;
    CK(run_moments(s));      // C of all components, FP64
    std::string err;
    if (!s->spectrum && (st = spectrum_create(s->geom, s->N, &s->spectrum, err)) != NFE_OK) return fail(st, "%s", err.c_str());
    if ((st = domain_size(s->spectrum, s->N, s->buf.fields, component, nbins, L, Sk, s->stream, err)) != NFE_OK)
        return fail(st, "%s", err.c_str());
    return NFE_OK;
}

nfe_status nfe_diagnostics(nfe_sim *s, nfe_diag *out) {
    nfe_status st = check_sim(s);
    if (st != NFE_OK) return st;
    if (!out) return fail(NFE_EINVAL, "out is NULL");
    if ((st = ensure_fields(s)) != NFE_OK) return st;
    const int N = s->N;
    CK(run_moments(s));
    CK(s->ops->reduce(s->geom, s->buf, s->buf.cur, kReduceBlocks, s->stream));
    std::vector<double> d(diag_count(N));
    CK(cudaMemcpyAsync(d.data(), s->buf.diag, d.size() * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    std::memset(out, 0, sizeof *out);
    out->step = s->step;
    out->N = N;
    for (int i = 0; i < N; ++i) {
        out->mass[i] = d[i];
        out->max_abs_C[i] = d[N + 9 + i];
        out->min_C[i] = d[2 * N + 9 + i];
    }
    for (int k = 0; k < 3; ++k) {
        out->momentum[k] = d[N + k];
        out->force_sum[k] = d[N + 3 + k];
        out->force_abs_sum[k] = d[N + 6 + k];
    }
    out->max_speed = d[3 * N + 9];
    out->nonfinite = d[3 * N + 10] != 0.0 ? 1 : 0;
    for (int i = 0; i < N; ++i) if (!std::isfinite(out->mass[i])) out->nonfinite = 1;
    return NFE_OK;
}

nfe_status nfe_get_info(const nfe_sim *s, nfe_info *out) {
    nfe_status st = check_sim(s);
    if (st != NFE_OK) return st;
    if (!out) return fail(NFE_EINVAL, "out is NULL");
    std::memset(out, 0, sizeof *out);
    out->lattice = s->grid.lattice;
    out->N = s->N;
    out->precision = s->prec;
    out->sites = s->geom.n;
    out->omega_stab = s->tab.omega;
    out->factor_residual = s->tab.residual;
    const int v = effective_variant(s, s->variant);
    out->kernels_per_step = (s->ops->vnk[v] > 0 ? s->ops->vnk[v] : s->ops->nk) + (s->buf.outflow ? 2 : 0);   // + the convective outflow
    out->variant = s->variant;
    out->nvariants = s->ops->nvariants;
    out->min_bytes_per_site = 2.0 * ((s->ops->Q - 1) * s->ops->f_elem_bytes + (s->N - 1) * s->ops->c_elem_bytes);
    if (s->buf.g[0]) out->min_bytes_per_site += 2.0 * (s->N - 1) * s->ops->Q * s->ops->c_elem_bytes;
    if (s->buf.node) out->min_bytes_per_site += 1.0;   // the node class
    out->state_bytes = state_size(s);
    out->device_bytes = s->device_bytes;
    return NFE_OK;
}

nfe_status nfe_get_state(nfe_sim *s, void *host, size_t bytes) {
    nfe_status st = check_sim(s);
    if (st != NFE_OK) return st;
    const size_t need = state_size(s);
    if (!host || bytes != need) return fail(NFE_EINVAL, "state buffer must be %zu bytes", need);
    char *h = static_cast<char *>(host);
    CK(cudaStreamSynchronize(s->stream));
    std::memcpy(h, &s->step, sizeof(int64_t));
    CK(cudaMemcpyAsync(h + sizeof(int64_t), s->buf.f[s->buf.cur], s->fplanes_bytes, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaMemcpyAsync(h + sizeof(int64_t) + s->fplanes_bytes, s->buf.C[s->buf.cur], s->cplanes_bytes,
                       cudaMemcpyDeviceToHost, s->stream));
    if (s->buf.g[0])
        CK(cudaMemcpyAsync(h + sizeof(int64_t) + s->fplanes_bytes + s->cplanes_bytes, s->buf.g[s->buf.cur],
                           s->gplanes_bytes, cudaMemcpyDeviceToHost, s->stream));
    if (s->ghost_bytes)
        CK(cudaMemcpyAsync(h + sizeof(int64_t) + s->fplanes_bytes + s->cplanes_bytes + s->gplanes_bytes,
                           s->buf.ghost[s->buf.cur], s->ghost_bytes, cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return NFE_OK;
}

nfe_status nfe_set_state(nfe_sim *s, const void *host, size_t bytes) {
    nfe_status st = check_sim(s);
    if (st != NFE_OK) return st;
    const size_t need = state_size(s);
    if (!host || bytes != need) return fail(NFE_EINVAL, "state buffer must be %zu bytes", need);
    const char *h = static_cast<const char *>(host);
    CK(cudaStreamSynchronize(s->stream));
    std::memcpy(&s->step, h, sizeof(int64_t));
    CK(cudaMemcpyAsync(s->buf.f[s->buf.cur], h + sizeof(int64_t), s->fplanes_bytes, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemcpyAsync(s->buf.C[s->buf.cur], h + sizeof(int64_t) + s->fplanes_bytes, s->cplanes_bytes,
                       cudaMemcpyHostToDevice, s->stream));
    if (s->buf.g[0])
        CK(cudaMemcpyAsync(s->buf.g[s->buf.cur], h + sizeof(int64_t) + s->fplanes_bytes + s->cplanes_bytes,
                           s->gplanes_bytes, cudaMemcpyHostToDevice, s->stream));
    if (s->ghost_bytes)
        CK(cudaMemcpyAsync(s->buf.ghost[s->buf.cur], h + sizeof(int64_t) + s->fplanes_bytes + s->cplanes_bytes + s->gplanes_bytes,
                           s->ghost_bytes, cudaMemcpyHostToDevice, s->stream));
    CK(cudaMemsetAsync(s->buf.flag, 0, sizeof(int), s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return NFE_OK;
}

nfe_status nfe_set_geometry(nfe_sim *s, const uint8_t *node, int ninlets, const double *inlets, int outflow) {
    nfe_status st = check_sim(s);
    if (st != NFE_OK) return st;
    CK(cudaStreamSynchronize(s->stream));
    for (auto &g : s->graph) if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    if (!node) {
        geo_free(s);
        return NFE_OK;
    }
    if (!s->ops->geo_prepare) return fail(NFE_EUNSUPPORTED, "no geometry form for this lattice");
    if (s->buf.g[0]) return fail(NFE_EUNSUPPORTED, "open and complex boundaries need tau_g = 1");
    if (s->no_phi) return fail(NFE_EUNSUPPORTED, "open and complex boundaries together with NFE_NO_PHI");
    if (ninlets < 0 || ninlets > kMaxInlets) return fail(NFE_EINVAL, "ninlets must be 0..%d", kMaxInlets);
    if (ninlets > 0 && !inlets) return fail(NFE_EINVAL, "inlets is NULL");
    const int N = s->N, nx = s->geom.nx, ny = s->geom.ny;
    const int D = s->ops->Q == 19 ? 3 : 2;           // velocity components of an inlet row
    const size_t n = size_t(s->geom.n);
    for (size_t i = 0; i < n; ++i)
        if (node[i] >= kNodeInlet0 + ninlets) return fail(NFE_EINVAL, "node class %d at site %zu (ninlets = %d)", int(node[i]), i, ninlets);
    // inlet rows in internal component order
    std::vector<double> rows(size_t(std::max(ninlets, 1)) * (D + N), 0.0);
    for (int j = 0; j < ninlets; ++j) {
        const double *r = inlets + size_t(j) * (D + N);
        double sum = 0.0;
        for (int a = 0; a < D + N; ++a)
            if (!std::isfinite(r[a])) return fail(NFE_EINVAL, "inlet %d: non-finite value", j);
        for (int a = 0; a < N; ++a) {
            if (r[D + a] < 0.0) return fail(NFE_EINVAL, "inlet %d: C_b[%d] < 0", j, a);
            sum += r[D + a];
        }
        if (std::fabs(sum - 1.0) > 1e-9) return fail(NFE_EINVAL, "inlet %d: C_b sums to %.17g, not 1", j, sum);
        double *o = rows.data() + size_t(j) * (D + N);
        for (int a = 0; a < D; ++a) o[a] = r[a];
        for (int a = 0; a < N; ++a) o[D + a] = r[D + s->uidx[a]];
    }
    const int nrows = ny * s->geom.nz;                // (y, z) lines of the grid
    if (outflow) {
        if (s->geom.wx) return fail(NFE_EINVAL, "outflow needs a periodic x axis (no x walls)");
        if (nx < 3) return fail(NFE_EINVAL, "outflow needs nx >= 3");
        for (int r = 0; r < nrows; ++r) {
            if (node[size_t(nx) * r] == kNodeFluid) return fail(NFE_EINVAL, "outflow: fluid node at (0, %d, %d)", r % ny, r / ny);
            if (node[size_t(nx) * r + nx - 1] >= kNodeInlet0)
                return fail(NFE_EINVAL, "outflow: inlet node at (%d, %d, %d)", nx - 1, r % ny, r / ny);
        }
    }
    geo_free(s);
    const size_t ce = s->ops->c_elem_bytes;
    if ((st = dev_alloc(s, reinterpret_cast<void **>(&s->node_dev), n)) != NFE_OK) return st;
    const size_t inl_row = size_t(2 * N + (D - 2));    // v_b (D), C_b and S_b of the evolved components
    if ((st = dev_alloc(s, &s->inl_dev, size_t(std::max(ninlets, 1)) * inl_row * ce)) != NFE_OK) { geo_free(s); return st; }
    if (outflow) {
        s->ghost_bytes = size_t(N - 1) * nrows * ce;
        for (int b = 0; b < 2; ++b)
            if ((st = dev_alloc(s, &s->buf.ghost[b], s->ghost_bytes)) != NFE_OK) { geo_free(s); return st; }
        const size_t pb = size_t(2 * ((nrows + 31) / 32)) * sizeof(double);   // 2 per CTA of the outflow (32 rows)
        if ((st = dev_alloc(s, reinterpret_cast<void **>(&s->buf.opart), pb)) != NFE_OK) { geo_free(s); return st; }
        s->geo_bytes += pb;
    }
    if (s->ops->Q == 19) {
        // the solid links of every site, formed once from the node classes
        if ((st = dev_alloc(s, reinterpret_cast<void **>(&s->buf.lmask), n * sizeof(unsigned))) != NFE_OK) { geo_free(s); return st; }
        s->geo_bytes += n * sizeof(unsigned);
    }
    s->geo_bytes += n + size_t(std::max(ninlets, 1)) * inl_row * ce + 2 * s->ghost_bytes;
    s->buf.node = s->node_dev;
    s->buf.inl = s->inl_dev;
    s->buf.outflow = outflow ? 1 : 0;
    s->ninlets = ninlets;
    cudaError_t e = cudaMemcpyAsync(s->node_dev, node, n, cudaMemcpyHostToDevice, s->stream);
    // the FP64 rows go through a small temporary device buffer
    void *rows_dev = nullptr;
    if (e == cudaSuccess && ninlets > 0) {
        const size_t rb = rows.size() * sizeof(double);
        if ((st = dev_alloc(s, &rows_dev, rb)) != NFE_OK) { geo_free(s); return st; }
        e = cudaMemcpyAsync(rows_dev, rows.data(), rb, cudaMemcpyHostToDevice, s->stream);
        if (e == cudaSuccess)
            e = s->ops->inlet_table(s->coef, static_cast<const double *>(rows_dev), ninlets, s->inl_dev, s->stream);
    }
    if (e == cudaSuccess) e = s->ops->geo_prepare(s->geom, s->buf, s->buf.cur, ninlets, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (rows_dev) {
        cudaStreamSynchronize(s->stream);
        dev_free(s, rows_dev);
        s->device_bytes -= rows.size() * sizeof(double);
    }
    if (e != cudaSuccess) { geo_free(s); return cuda_fail(e, "nfe_set_geometry"); }
    return NFE_OK;
}

nfe_status nfe_set_variant(nfe_sim *s, int variant) {
    nfe_status st = check_sim(s);
    if (st != NFE_OK) return st;
    if (variant >= s->ops->nvariants) return fail(NFE_EINVAL, "variant %d >= %d", variant, s->ops->nvariants);
    CK(cudaStreamSynchronize(s->stream));
    for (auto &g : s->graph) if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    s->variant = variant < 0 ? -1 : variant;
    return NFE_OK;
}

nfe_status nfe_profile_enable(nfe_sim *s, int on) {
    nfe_status st = check_sim(s);
    if (st != NFE_OK) return st;
    CK(cudaStreamSynchronize(s->stream));
    for (auto &t : s->timed) { s->event_pool.push_back(t.a); s->event_pool.push_back(t.b); }
    s->timed.clear();
    for (int k = 0; k < K_NKINDS; ++k) { s->prof_launches[k] = 0; s->prof_ms[k] = 0.0; }
    s->profiling = on != 0;
    return NFE_OK;
}

nfe_status nfe_profile_read(nfe_sim *s, int max_kinds, int *kinds, const char **names,
                            int64_t *launches, double *total_ms) {
    nfe_status st = check_sim(s);
    if (st != NFE_OK) return st;
    if (!kinds) return fail(NFE_EINVAL, "kinds is NULL");
    CK(cudaStreamSynchronize(s->stream));
    for (auto &t : s->timed) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, t.a, t.b));
        s->prof_launches[t.kind] += 1;
        s->prof_ms[t.kind] += ms;
        s->event_pool.push_back(t.a);
        s->event_pool.push_back(t.b);
    }
    s->timed.clear();
    int c = 0;
    for (int k = 0; k < K_NKINDS && c < max_kinds; ++k) {
        if (s->prof_launches[k] == 0) continue;
        if (names) names[c] = kKernelNames[k];
        if (launches) launches[c] = s->prof_launches[k];
        if (total_ms) total_ms[c] = s->prof_ms[k];
        ++c;
    }
    *kinds = c;
    return NFE_OK;
}

nfe_status nfe_bulk_potential_host(int N, const double *sigma, double D, double omega_stab,
                                   int implicit_component, int npts, const double *Cpts, double *S) {
    if (N < 2 || N > NFE_MAX_N) return fail(NFE_EINVAL, "N = %d outside 2..%d", N, NFE_MAX_N);
    if (!sigma || !Cpts || !S || npts < 0) return fail(NFE_EINVAL, "NULL argument or npts < 0");
    if (!(D > 0.0)) return fail(NFE_EINVAL, "D must be positive");
    if (implicit_component < 0 || implicit_component >= N) return fail(NFE_EINVAL, "implicit_component out of range");
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            if ((i == j && sigma[i * N + j] != 0.0) || (i != j && !(sigma[i * N + j] > 0.0)) ||
                sigma[i * N + j] != sigma[j * N + i])
                return fail(NFE_EINVAL, "sigma must be symmetric, zero on the diagonal, positive elsewhere");
    int uidx[NFE_MAX_N];
    int a = 0;
    for (int c = 0; c < N; ++c) if (c != implicit_component) uidx[a++] = c;
    uidx[N - 1] = implicit_component;
    const double omega = std::isnan(omega_stab) ? (auto_omega(N, sigma) ? 1.0 / 90.0 : 0.0) : omega_stab;
    Tables tab;
    std::string err;
    nfe_status st = build_tables(N, sigma, uidx, D, omega, true, tab, err);
    if (st != NFE_OK) return fail(st, "%s", err.c_str());
    const int m2 = N * (N + 1) / 2, m4 = mono4s_count(N);
    for (int p = 0; p < npts; ++p) {
        double c[NFE_MAX_N];
        for (int k = 0; k < N; ++k) c[k] = Cpts[size_t(p) * N + uidx[k]];
        double *out = S + size_t(p) * N;
        out[implicit_component] = 0.0;
        for (int e = 0; e < N - 1; ++e) {
            double q = 0.0;
            int idx = 0;
            for (int i = 0; i < N; ++i)
                for (int j = i; j < N; ++j) q += tab.q2[e * m2 + idx++] * c[i] * c[j];
            if (!tab.q4.empty()) {
                // structured quartic part, in the layout of the table (see nfe_internal.h)
                const double *a4 = tab.q4.data() + e * m4;
                int jdx = 0;
                double sa = 0.0, sb = 0.0;
                for (int l = 0; l < N; ++l) {
                    if (l == e) continue;
                    double lin = 0.0;
                    for (int m = 0; m < N; ++m) if (m != e && m != l) lin += a4[jdx++] * c[m];
                    sa += c[l] * c[l] * lin;
                }
                for (int k = 0; k < N; ++k)
                    for (int l = k + 1; l < N; ++l)
                        if (k != e && l != e) sb += a4[jdx++] * c[k] * c[k] * c[l] * c[l];
                q += c[e] * sa + sb;
            }
            out[uidx[e]] = c[e] * q;
        }
    }
    return NFE_OK;
}

}  // extern "C"

// ============================================================================
// Batched sweep (nfe_batch_*): many nfe_sim advanced by one persistent launch
// ============================================================================

struct nfe_batch {
    int nsims = 0;
    int prec = 0;
    std::vector<nfe_sim *> sims;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    const BatchOps *ops = nullptr;
    void *d_sims = nullptr;           // BatchSim<T>[nsims]
    size_t sim_bytes = 0;             // sizeof(BatchSim<T>)
    int4 *d_items = nullptr;
    size_t items_cap = 0;
    BatchSync *d_sync = nullptr;
    int variant = -1;
    int grid = 0;
    int nitems = 0;
    int nstart[kBatchGroups] = {0};     // work-list range of each (N, form) group
    int ncount[kBatchGroups] = {0};
    bool forms = false;                 // some member runs the no-phi or the stored-population form
    int parity = 0;
    int mode = NFE_BATCH_AUTO;        // requested form
    int form = -1;                    // form in use (persistent or per-step) after tuning
    long long spin_default = 20000000LL;   // polls (~100 ns each plus the poll itself)
    long long spin_next = 0;               // test hook: limit for the next launch
    unsigned extra_next = 0;               // test hook: phantom CTAs for the next launch
    int64_t sites = 0;
    bool graphs_ok = true;
    std::map<std::pair<int64_t, int>, cudaGraphExec_t> graphs;
};

namespace {

// form of a member's step (kBatchForms)
int batch_form(const nfe_sim *s) { return s->buf.g[0] ? 2 : (s->no_phi ? 1 : 0); }

template <typename T>
void fill_batch_sim(const nfe_sim *s, BatchSim<T> &d) {
    std::memset(&d, 0, sizeof d);
    d.geom = s->geom;
    d.N = s->N;
    d.form = batch_form(s);
    d.coef = *static_cast<const Coef<T> *>(s->coef);
    d.f[0] = s->buf.f[0];
    d.f[1] = s->buf.f[1];
    d.C[0] = s->buf.C[0];
    d.C[1] = s->buf.C[1];
    d.g[0] = s->buf.g[0];
    d.g[1] = s->buf.g[1];
    d.flag = s->buf.flag;
}

nfe_status upload_batch_sim(nfe_batch *b, int i) {
    std::vector<unsigned char> tmp(b->sim_bytes);
    if (b->prec == NFE_FP64) fill_batch_sim<double>(b->sims[i], *reinterpret_cast<BatchSim<double> *>(tmp.data()));
    else fill_batch_sim<float>(b->sims[i], *reinterpret_cast<BatchSim<float> *>(tmp.data()));
    CK(cudaMemcpyAsync(static_cast<char *>(b->d_sims) + size_t(i) * b->sim_bytes, tmp.data(), b->sim_bytes,
                       cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    return NFE_OK;
}

nfe_status batch_items(nfe_batch *b, int v) {
    const int TX = 32, TY = b->ops->ty[v];
    // simulations grouped by component count and form: CTAs that run at the same time then
    // execute the same tile code (one unrolled body per N), which keeps the instruction cache
    // warm (grouping further by walls or Omega measured no difference)
    auto group = [&](int i) { return (b->sims[i]->N - 2) * kBatchForms + batch_form(b->sims[i]); };
    std::vector<int> order(b->nsims);
    for (int i = 0; i < b->nsims; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return group(a) < group(c); });
    std::vector<int4> items;
    for (int q = 0; q < kBatchGroups; ++q) { b->nstart[q] = 0; b->ncount[q] = 0; }
    for (int i : order) {
        const Geom &g = b->sims[i]->geom;
        const int grp = group(i);
        if (b->ncount[grp] == 0) b->nstart[grp] = int(items.size());
        for (int y0 = 0; y0 < g.ny; y0 += TY)
            for (int x0 = 0; x0 < g.nx; x0 += TX) {
                items.push_back(make_int4(i, x0, y0, 0));
                ++b->ncount[grp];
            }
    }
    if (items.size() > b->items_cap) {
        if (b->d_items) cudaFree(b->d_items);
        b->d_items = nullptr;
        cudaError_t e = cudaMalloc(&b->d_items, items.size() * sizeof(int4));
        if (e != cudaSuccess) { cudaGetLastError(); return fail(NFE_ENOMEM, "batch work list: %s", cudaGetErrorString(e)); }
        b->items_cap = items.size();
    }
    CK(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    b->nitems = int(items.size());
    int bps = 0;
    CK(b->ops->setup[v](&bps));
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (bps < 1) return fail(NFE_EUNSUPPORTED, "batched kernel does not fit on an SM");
    b->grid = std::min(bps * sms, b->nitems);
    return NFE_OK;
}

BatchLaunch batch_launch_args(const nfe_batch *b, int64_t nsteps, long long spins, unsigned extra) {
    BatchLaunch L;
    L.sims = b->d_sims;
    L.items = b->d_items;
    L.nitems = b->nitems;
    L.nsteps = int(nsteps);
    L.parity = b->parity;
    L.sync = b->d_sync;
    L.spin_limit = spins;
    L.expected = unsigned(b->grid) + extra;
    L.grid = b->grid;
    for (int q = 0; q < kBatchGroups; ++q) { L.nstart[q] = b->nstart[q]; L.ncount[q] = b->ncount[q]; }
    return L;
}

// Time every (launch form, tile shape) the requested mode allows on the current
// state and keep the fastest.  One step reads buffer `parity` and writes the
// other one, so the state is untouched.
nfe_status batch_autotune(nfe_batch *b) {
    if (b->variant >= 0) return NFE_OK;
    {
        // a timeout still to be reported by nfe_batch_sync: the trial launches would clear it
        BatchSync sync;
        CK(cudaStreamSynchronize(b->stream));
        CK(cudaMemcpy(&sync, b->d_sync, sizeof sync, cudaMemcpyDeviceToHost));
        if (sync.error) return fail(NFE_ETIMEOUT, "a grid-barrier wait of the batched kernel ran out of spins");
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = 1e300;
    int best_v = 0, best_form = NFE_BATCH_PERSISTENT;
    for (int form = NFE_BATCH_PERSISTENT; form <= NFE_BATCH_PER_STEP; ++form) {
        if (b->mode != NFE_BATCH_AUTO && b->mode != form) continue;
        // members with the no-phi or stored-population form: per-step launches on 32 x 8 tiles
        if (b->forms && form == NFE_BATCH_PERSISTENT) continue;
        for (int v = 0; v < kBatchVariants; ++v) {
            if (b->forms && b->ops->ty[v] != 8) continue;
            nfe_status st = batch_items(b, v);
            if (st != NFE_OK) return st;
            BatchLaunch L = batch_launch_args(b, 1, b->spin_default, 0);
            const BatchLauncher launch = form == NFE_BATCH_PERSISTENT ? b->ops->persistent[v] : b->ops->per_step[v];
            CK(cudaMemsetAsync(b->d_sync, 0, sizeof(BatchSync), b->stream));
            CK(launch(L, b->stream));
            CK(cudaEventRecord(e0, b->stream));
            for (int r = 0; r < 3; ++r) {
                CK(cudaMemsetAsync(b->d_sync, 0, sizeof(BatchSync), b->stream));
                CK(launch(L, b->stream));
            }
            CK(cudaEventRecord(e1, b->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.0f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; best_v = v; best_form = form; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    nfe_status st = batch_items(b, best_v);
    if (st != NFE_OK) return st;
    for (nfe_sim *s : b->sims) CK(cudaMemsetAsync(s->buf.flag, 0, sizeof(int), b->stream));
    b->variant = best_v;
    b->form = best_form;
    return NFE_OK;
}

void batch_free(nfe_batch *b) {
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    for (nfe_sim *s : b->sims) {
        if (!s) continue;
        s->stream = nullptr;          // the batch owns the stream
        s->own_stream = false;
        free_all(s);
        delete s;
    }
    b->sims.clear();
    if (b->d_sims) cudaFree(b->d_sims);
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_sync) cudaFree(b->d_sync);
    b->d_sims = nullptr;
    b->d_items = nullptr;
    b->d_sync = nullptr;
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    b->stream = nullptr;
}

}  // namespace

extern "C" {

nfe_status nfe_batch_create(int nsims, const nfe_grid *grids, const int *N, const nfe_params *params,
                            nfe_batch **out) {
    if (!out) return fail(NFE_EINVAL, "out is NULL");
    *out = nullptr;
    if (nsims < 1 || !grids || !N || !params) return fail(NFE_EINVAL, "nsims < 1 or NULL array");
    const int prec = params[0].precision;
    if (prec != NFE_FP32 && prec != NFE_FP64)
        return fail(NFE_EUNSUPPORTED, "batched sweeps run in NFE_FP32 or NFE_FP64");
    for (int i = 0; i < nsims; ++i) {
        if (grids[i].lattice != NFE_D2Q9) return fail(NFE_EUNSUPPORTED, "batched sweeps are D2Q9 (simulation %d)", i);
        if (N[i] < 2 || N[i] > 5) return fail(NFE_EUNSUPPORTED, "batched sweeps take N = 2..5 (simulation %d)", i);
        if (params[i].precision != prec) return fail(NFE_EINVAL, "all simulations of a batch share one precision");
    }
    nfe_batch *b = new (std::nothrow) nfe_batch();
    if (!b) return fail(NFE_ENOMEM, "host allocation failed");
    b->nsims = nsims;
    b->prec = prec;
    b->ops = batch_ops(prec);
    if (params[0].cuda_stream) {
        b->stream = static_cast<cudaStream_t>(params[0].cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreate(&b->stream);
        if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaStreamCreate"); }
        b->own_stream = true;
    }
    b->sims.assign(nsims, nullptr);
    for (int i = 0; i < nsims; ++i) {
        nfe_params p = params[i];
        p.cuda_stream = b->stream;
        nfe_status st = nfe_create(&grids[i], N[i], &p, &b->sims[i]);
        if (st != NFE_OK) {
            std::string msg = g_err;
            batch_free(b);
            delete b;
            return fail(st, "simulation %d: %s", i, msg.c_str());
        }
        b->sites += b->sims[i]->geom.n;
        if (batch_form(b->sims[i]) != 0) b->forms = true;
    }
    b->sim_bytes = prec == NFE_FP64 ? sizeof(BatchSim<double>) : sizeof(BatchSim<float>);
    cudaError_t e = cudaMalloc(&b->d_sims, b->sim_bytes * nsims);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_sync, sizeof(BatchSync));
    if (e != cudaSuccess) { cudaGetLastError(); batch_free(b); delete b; return fail(NFE_ENOMEM, "batch descriptors"); }
    for (int i = 0; i < nsims; ++i) {
        nfe_status st = upload_batch_sim(b, i);
        if (st != NFE_OK) { batch_free(b); delete b; return st; }
    }
    e = cudaMemsetAsync(b->d_sync, 0, sizeof(BatchSync), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) { batch_free(b); delete b; return cuda_fail(e, "batch init"); }
    *out = b;
    return NFE_OK;
}

void nfe_batch_destroy(nfe_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free(b);
    delete b;
}

nfe_status nfe_batch_set_fields(nfe_batch *b, int sim, const double *C, const double *v) {
    if (!b || sim < 0 || sim >= b->nsims) return fail(NFE_EINVAL, "bad batch or simulation index");
    nfe_sim *s = b->sims[sim];
    nfe_status st = nfe_set_fields(s, C, v);          // state in buffer 0
    if (st != NFE_OK) return st;
    if (b->parity == 1) {
        // the batch's current buffer is 1 for every simulation: swap this one's buffers
        std::swap(s->buf.f[0], s->buf.f[1]);
        std::swap(s->buf.C[0], s->buf.C[1]);
        std::swap(s->buf.g[0], s->buf.g[1]);
        s->buf.cur = 1;
        for (auto &g : s->graph) if (g) { cudaGraphExecDestroy(g); g = nullptr; }
        return upload_batch_sim(b, sim);
    }
    return NFE_OK;
}

nfe_status nfe_batch_set_mode(nfe_batch *b, int mode) {
    if (!b || (mode != NFE_BATCH_PERSISTENT && mode != NFE_BATCH_PER_STEP && mode != NFE_BATCH_AUTO))
        return fail(NFE_EINVAL, "bad mode");
    if (mode == NFE_BATCH_PERSISTENT && b->forms)
        return fail(NFE_EUNSUPPORTED, "the persistent form runs members without NFE_NO_PHI and with tau_g = 1");
    CK(cudaStreamSynchronize(b->stream));
    b->mode = mode;
    b->variant = -1;                 // re-tune for the new mode
    b->form = -1;
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    return NFE_OK;
}

nfe_status nfe_batch_set_barrier_test(nfe_batch *b, int64_t spins, int extra) {
    if (!b || extra < 0) return fail(NFE_EINVAL, "bad arguments");
    if (b->forms) return fail(NFE_EUNSUPPORTED, "the barrier test runs the persistent form");
    b->spin_next = spins > 0 ? spins : 0;
    b->extra_next = unsigned(extra);
    return NFE_OK;
}

nfe_status nfe_batch_step(nfe_batch *b, int64_t nsteps) {
    if (!b) return fail(NFE_EINVAL, "batch is NULL");
    if (nsteps < 0 || nsteps > (1LL << 30)) return fail(NFE_EINVAL, "nsteps out of range");
    if (nsteps == 0) return NFE_OK;
    nfe_status st = batch_autotune(b);
    if (st != NFE_OK) return st;
    const int v = b->variant;
    if (b->spin_next > 0 || b->extra_next > 0) {
        // fault-injection launch (direct, not captured)
        BatchLaunch L = batch_launch_args(b, nsteps, b->spin_next > 0 ? b->spin_next : b->spin_default, b->extra_next);
        CK(cudaMemsetAsync(b->d_sync, 0, kBatchSyncResetBytes, b->stream));
        CK(b->ops->persistent[v](L, b->stream));
        b->spin_next = 0;
        b->extra_next = 0;
    } else {
        const auto key = std::make_pair(nsteps, b->parity);
        auto it = b->graphs.find(key);
        if (it == b->graphs.end() && b->graphs_ok) {
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ex = nullptr;
            BatchLaunch L = batch_launch_args(b, nsteps, b->spin_default, 0);
            const BatchLauncher launch = b->form == NFE_BATCH_PER_STEP ? b->ops->per_step[v] : b->ops->persistent[v];
            cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e1 = cudaMemsetAsync(b->d_sync, 0, kBatchSyncResetBytes, b->stream);
                cudaError_t e2 = e1 == cudaSuccess ? launch(L, b->stream) : e1;
                e = cudaStreamEndCapture(b->stream, &g);
                if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
                else if (e == cudaSuccess) e = e2;
                if (g) cudaGraphDestroy(g);
            }
            if (e == cudaSuccess && ex) {
                it = b->graphs.emplace(key, ex).first;
            } else {
                cudaGetLastError();
                b->graphs_ok = false;          // cooperative launches not capturable: launch directly
            }
        }
        if (it != b->graphs.end()) {
            CK(cudaGraphLaunch(it->second, b->stream));
        } else {
            BatchLaunch L = batch_launch_args(b, nsteps, b->spin_default, 0);
            CK(cudaMemsetAsync(b->d_sync, 0, kBatchSyncResetBytes, b->stream));
            CK((b->form == NFE_BATCH_PER_STEP ? b->ops->per_step[v] : b->ops->persistent[v])(L, b->stream));
        }
    }
    b->parity ^= int(nsteps & 1);
    for (nfe_sim *s : b->sims) {
        s->buf.cur = b->parity;
        s->step += nsteps;
    }
    return NFE_OK;
}

nfe_status nfe_batch_sync(nfe_batch *b) {
    if (!b) return fail(NFE_EINVAL, "batch is NULL");
    CK(cudaStreamSynchronize(b->stream));
    BatchSync sync;
    CK(cudaMemcpy(&sync, b->d_sync, sizeof sync, cudaMemcpyDeviceToHost));
    if (sync.error) {
        // reported once: the error word is cleared, the state stays undefined until set_fields
        CK(cudaMemset(&b->d_sync->error, 0, sizeof(int)));
        return fail(NFE_ETIMEOUT, "a grid-barrier wait of the batched kernel ran out of spins");
    }
    for (int i = 0; i < b->nsims; ++i) {
        int flag = 0;
        CK(cudaMemcpy(&flag, b->sims[i]->buf.flag, sizeof(int), cudaMemcpyDeviceToHost));
        if (flag) return fail(NFE_ENONFINITE, "simulation %d: a volume fraction became NaN or Inf", i);
    }
    return NFE_OK;
}

nfe_status nfe_batch_fields(nfe_batch *b, int sim, double *C, double *v, double *P) {
    if (!b || sim < 0 || sim >= b->nsims) return fail(NFE_EINVAL, "bad batch or simulation index");
    return nfe_fields(b->sims[sim], C, v, P);
}

nfe_status nfe_batch_diagnostics(nfe_batch *b, int sim, nfe_diag *out) {
    if (!b || sim < 0 || sim >= b->nsims) return fail(NFE_EINVAL, "bad batch or simulation index");
    return nfe_diagnostics(b->sims[sim], out);
}

nfe_status nfe_batch_get_info(const nfe_batch *b, nfe_batch_info *out) {
    if (!b || !out) return fail(NFE_EINVAL, "NULL argument");
    std::memset(out, 0, sizeof *out);
    out->nsims = b->nsims;
    out->sites = b->sites;
    out->nitems = b->nitems;
    out->grid = b->grid;
    out->tile_x = b->variant >= 0 ? 32 : 0;
    out->tile_y = b->variant >= 0 ? b->ops->ty[b->variant] : 0;
    out->graphs = (b->graphs_ok && !b->graphs.empty()) ? 1 : 0;
    out->form = b->form;
    return NFE_OK;
}

}  // extern "C"
