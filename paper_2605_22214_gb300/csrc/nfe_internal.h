// Internal interface between the host side (nfe_host.cpp) and the kernels
// (nfe_kernels.cuh, instantiated per lattice in nfe_d2q9.cu / nfe_d3q19.cu).
// Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nfe.h"

namespace nfe {

constexpr int kMaxN = NFE_MAX_N;
constexpr int kMaxMono2 = kMaxN * (kMaxN + 1) / 2;   // degree-2 monomials in 8 variables

// Coefficients of the quartic (stabiliser) part of q_i per evolved component i, structured as
//   C_i sum_{l != i} C_l^2 sum_{m not in {i,l}} a_{ilm} C_m + sum_{k<l; i not in {k,l}} b_{ikl} C_k^2 C_l^2:
// (N-1)(N-2) values a, then (N-1)(N-2)/2 values b.
__host__ __device__ constexpr int mono4s_count(int n) { return 3 * (n - 1) * (n - 2) / 2; }

// Degree-3 monomials a <= b <= c over the N - 1 components other than i: the part of the bulk
// flux potential that is not divisible by C_i once phi_j is dropped (the no-phi ablation).
__host__ __device__ constexpr int mono3r_count(int n) { return (n - 1) * n * (n + 1) / 6; }

// Up to N = 6 the quartic coefficients also travel with the kernel parameters (constant bank).
constexpr int kQ4InlineMaxN = 6;
constexpr int kQ4Inline = (kQ4InlineMaxN - 1) * mono4s_count(kQ4InlineMaxN);   // 150

// Grid geometry as the kernels see it.
struct Geom {
    int nx, ny, nz;
    int wx, wy, wz;       // 1 = halfway walls on that axis
    long long n;          // nx * ny * nz
};

// Per-simulation coefficients, passed to the kernels by value.  Components are
// in the internal order: the evolved components first (in the user's order),
// the implicit one last (slot N-1).
template <typename T>
struct Coef {
    T beta[kMaxN][kMaxN];         // beta_ab = 6 sigma_ab / D (Sec. II)
    T kappa[kMaxN][kMaxN];        // kappa_ab = 3 D sigma_ab / 4
    T q2[kMaxN - 1][kMaxMono2];   // factored flux potential, degree-2 part, per evolved slot
    T omp[kMaxN];                 // omega+ of each component (1 / tau_i)
    T omm[kMaxN];                 // omega- of each component (Eq. 26, or omega+ for BGK)
    int uidx[kMaxN];              // user index of each internal slot (argmax ties -> lowest)
    T m;                          // g^eq coefficient m (Eq. 40)
    T d34;                        // 3 D / 4
    T fb[3];                      // body force
    T fscale;                     // FP16 storage scale 2^scale_exp (1 otherwise)
    T finv;                       // 1 / fscale
    int has_q4;                   // Omega != 0: degree-4 part present
    int nonconservative;          // force of Eq. 31 instead of Eq. 34
    const T *q4;                  // (N-1) x mono4s_count(N), device memory, or nullptr (Omega = 0)
    const T *r3;                  // (N-1) x mono3r_count(N), device memory: no-phi remainder, or nullptr
    int no_phi;                   // the no-phi ablation (flux potential without phi_j)
    T gomega;                     // 1 / tau_g (stored-g path, tau_g != 1)
    int has_fc;                   // body force on one component present
    int uniform_tau;              // every component has the same omega+ and omega- (Eq. 42 has no choice)
    T fc[3];                      // that force per unit volume fraction, F += C_c F_c
    T fcsel[kMaxN];               // 1 for the internal slot of component c, 0 elsewhere
    T q4c[kQ4Inline];             // the same coefficients in the parameter block (N <= 6); last member
};

// Node classes of the D2Q9 geometry (open and complex boundaries, Sec. III C): one byte per
// site.  Inside the kernels, kNodeGhost marks the outflow ghost column beyond x = nx - 1.
constexpr unsigned char kNodeFluid = 0, kNodeSolid = 1, kNodeInlet0 = 2, kNodeGhost = 255;
constexpr int kMaxInlets = 64;

// One kernel kind for profiling.
// K_PHYS / K_GATHER: the two kernels of the split D3Q19 step.
enum KernelKind { K_FUSED = 0, K_MOMENTS = 1, K_REDUCE = 2, K_PHYS = 3, K_GATHER = 4, K_NKINDS = 5 };
extern const char *kKernelNames[K_NKINDS];

// Device buffers of one simulation.
struct Buffers {
    void *f[2];           // populations k = 1..Q-1, planar, storage type
    void *C[2];           // evolved volume fractions, planar, compute type
    void *g[2];           // component populations ((N-1) x Q planes, compute type) when tau_g != 1, else null
    double *fields;       // moments output: C (N), v (3), P, Fs (3) planes, FP64
    double *partials;     // reduction partials
    double *diag;         // reduction result
    int *flag;            // non-finite flag
    int cur;              // index of the buffer holding the current state
    // geometry (null when the grid has none)
    const unsigned char *node;   // node class per site
    const void *inl;             // inlet table, compute type: per inlet vx, vy, C_b (N-1), S_b (N-1)
    void *ghost[2];              // outflow ghost column, (N-1) x (ny nz), compute type, or null
    int outflow;                 // convective outflow on the x = nx - 1 edge
    double *opart;               // outflow partial sums (2 per 32 rows), or null
    unsigned *lmask;             // D3Q19 geometry: per site, bit k set when x + e_k is a solid node
                                 // (k = 1..18) and bit 31 when x is; or null
    void *vs;                    // split D3Q19 step: per-site gather records (C, v, S of the evolved
                                 // components, 2N - 1 + 2 values), compute type, or null
};

// Launchers exported by the lattice translation units.  Each returns
// cudaSuccess or the launch error.
using StepKernel = cudaError_t (*)(const Geom &, const void *coef, const Buffers &, int cur, cudaStream_t,
                                   int variant);
constexpr int kMaxVariants = 4;
struct Ops {
    int Q, D, N, prec;
    // one time step = nk kernels, state in buffers cur -> 1 - cur (cur is not flipped);
    // `variant` selects a tile shape (0 .. nvariants-1)
    int nk;
    int kinds[2];
    StepKernel kern[2];
    int nvariants;
    const char *variant_names[kMaxVariants];
    // fields (C, v, P, Fs in FP64) of the state in buffer cur
    cudaError_t (*moments)(const Geom &, const void *coef, const Buffers &, int cur, cudaStream_t);
    // FP64 reductions of bufs.fields (+ f and C finiteness) into bufs.diag
    cudaError_t (*reduce)(const Geom &, const Buffers &, int cur, int nblocks, cudaStream_t);
    // f = f^eq(P = 0, v) from an FP64 device velocity array (3 x n)
    cudaError_t (*init_f)(const Geom &, const void *coef, const Buffers &, int cur, const double *v, cudaStream_t);
    // populations of buffer cur to FP64 ((Q-1) x n, device)
    cudaError_t (*unpack_f)(const Geom &, const void *coef, const Buffers &, int cur, double *out, cudaStream_t);
    // evolved C from FP64 device array ((N-1) x n) into buffer cur
    cudaError_t (*pack_C)(const Geom &, const Buffers &, int cur, const double *in, cudaStream_t);
    // g = g^eq(C, v, S(C)) in buffer cur from C of buffer cur and an FP64 velocity (3 x n, or null)
    cudaError_t (*init_g)(const Geom &, const void *coef, const Buffers &, int cur, const double *v, cudaStream_t);
    int f_elem_bytes;     // bytes per stored population
    int c_elem_bytes;     // bytes per stored volume fraction (and per scratch value)
    // geometry: the inlet table from FP64 rows (vx, vy, C_b of all N components in internal
    // order) on the device (D2Q9; null for D3Q19, which takes fluid and solid nodes only);
    // C := C_b on the inlet nodes and ghost := column nx - 1 in buffer cur; the fields of the
    // state in buffer cur with the node classes
    cudaError_t (*inlet_table)(const void *coef, const double *rows, int ninl, void *out, cudaStream_t);
    cudaError_t (*geo_prepare)(const Geom &, const Buffers &, int cur, int ninl, cudaStream_t);
    cudaError_t (*moments_geo)(const Geom &, const void *coef, const Buffers &, int cur, cudaStream_t);
    // variants whose step is a different number of kernels (0: nk and kinds above): kern[0 ..
    // vnk[v] - 1] with kinds vkinds[v]
    int vnk[kMaxVariants];
    int vkinds[kMaxVariants][2];
    int scratch_planes;   // planes of the compute type per site for Buffers::vs (0: none)
};

// One translation unit per lattice and precision (compiled in parallel).
const Ops *ops_d2q9_fp64(int N);
const Ops *ops_d2q9_fp32(int N);
const Ops *ops_d2q9_f16(int N);
const Ops *ops_d2q9_bf16(int N);
const Ops *ops_d3q19_fp64(int N);
const Ops *ops_d3q19_fp32(int N);
const Ops *ops_d3q19_f16(int N);
const Ops *ops_d3q19_bf16(int N);

// Number of values one reduction block writes (and the diag layout):
//  [0, N) mass, [N, N+3) momentum, [N+3, N+6) force sum, [N+6, N+9) |force| sum,
//  [N+9, 2N+9) max |C|, [2N+9, 3N+9) min C, 3N+9 max speed, 3N+10 nonfinite.
__host__ __device__ constexpr int diag_count(int N) { return 3 * N + 11; }

// Records `msg` as the calling thread's last error (nfe_last_error) and returns s.
nfe_status set_error(nfe_status s, const char *msg);
constexpr int kReduceBlocks = 1024;

}  // namespace nfe
