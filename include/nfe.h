/*
 * nfe.h -- C ABI of the N-component free-energy lattice Boltzmann library
 * (arXiv 2605.22214, Rennick, Zhang, Bingert, Krause and Kusumaatmaja),
 * built for one NVIDIA GB300 (sm_103a).
 *
 * The library advances, on one GPU, the per-time-step lattice update of the
 * paper's method for N immiscible components:
 *   - isotropic gradients and Laplacians of the volume fractions C_i
 *     (Sec. III A, Eqs. 35-36), the chemical potentials (Sec. II, Eq. 7) and
 *     the reduction-consistent flux potential
 *     S_i = sum_j alpha_ij (mu_j + phi_j + xi_j)          (Sec. II, Eqs. 8-19),
 *   - the momentum-conserving surface-tension force
 *     F_s = grad E_B + sum_{i != j} kappa_ij lap C_j grad C_i  (Sec. III A, Eq. 34),
 *   - TRT collision with forcing and streaming of the hydrodynamic populations
 *     f_k on D2Q9 or D3Q19 (Sec. III A, Eqs. 22-30, 37-38), and the
 *     Cahn-Hilliard lattice Boltzmann update of the N-1 evolved volume
 *     fractions (Sec. III B, Eqs. 39-43): with tau_g = 1 collapsed onto C (no
 *     stored component populations), or with the populations stored for any
 *     other tau_g (nfe_params.tau_g),
 *   - halfway bounce-back and the wall-gradient rule on walls, periodic
 *     wrap on every other edge (Sec. III C, Eqs. 44-45);
 *   - solid nodes anywhere in the grid, velocity and volume-fraction inlets and the
 *     convective outflow, on D2Q9 and D3Q19 (Sec. III C; nfe_set_geometry).
 *
 * Conventions shared by every call:
 *   - Site index s = x + nx * (y + ny * z), x fastest.  Field arrays are
 *     planar: component c of site s sits at [c * n + s], n = nx * ny * nz.
 *   - Components are numbered 0 .. N-1 (the paper counts 1 .. N).  One of them,
 *     `implicit_component`, is not evolved: C_implicit = 1 - sum of the others
 *     (Sec. II, below Eq. 3).  An absent component that must stay exactly 0.0
 *     has to be an evolved one.
 *   - The library owns all device memory it allocates (cudaMalloc at create,
 *     cudaFree at destroy, or the caller's hooks in nfe_params).  Host buffers passed in are read or written
 *     during the call only and remain the caller's.
 *   - Every call returns an nfe_status; none throws, aborts or exits.
 *     nfe_last_error() gives a one-line message for the last failure on the
 *     calling thread.
 *   - Work is queued on the stream given in nfe_params.cuda_stream (borrowed;
 *     NULL = the legacy default stream).  nfe_step is asynchronous; the calls
 *     that return data to the host synchronise that stream.
 */
#ifndef NFE_H
#define NFE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NFE_OK = 0,
    NFE_EINVAL = 1,        /* an argument is out of range or inconsistent */
    NFE_ENOMEM = 2,        /* device or host allocation failed */
    NFE_ECUDA = 3,         /* a CUDA runtime call failed (message in nfe_last_error) */
    NFE_ESINGULAR = 4,     /* the alpha, Lambda or Theta system (Eqs. 8-19) has no unique solution */
    NFE_ENONFINITE = 5,    /* a kernel produced a NaN or Inf volume fraction */
    NFE_ETIMEOUT = 6,      /* a device-side wait of the batched kernel ran out of spins */
    NFE_EUNSUPPORTED = 7   /* a valid combination the library does not implement */
} nfe_status;

enum { NFE_D2Q9 = 9, NFE_D3Q19 = 19 };

enum {
    NFE_FP64 = 0,             /* all state and arithmetic in FP64 */
    NFE_FP32 = 1,             /* f and C stored and computed in FP32 */
    NFE_FP32_F16STORE = 2,    /* f stored as FP16 f_k / w_k * 2^scale_exp, arithmetic FP32 */
    NFE_FP32_BF16STORE = 3    /* f stored as BF16 f_k / w_k, arithmetic FP32 */
};

enum { NFE_WALL_X = 1, NFE_WALL_Y = 2, NFE_WALL_Z = 4 };

/* Flags (nfe_params.flags). */
enum {
    NFE_NONCONSERVATIVE_FORCE = 1,  /* F_s = sum_i mu_i grad C_i (Eq. 31) instead of Eq. 34 */
    NFE_NO_PHI = 2                  /* drop phi_j from the flux potential (Eq. 12): the ablation in
                                       which an absent component nucleates at interfaces (Sec. IV).
                                       D3Q19: the split form of the step; batches: per-step
                                       launches on 32 x 8 tiles (nfe_batch_set_mode) */
};

#define NFE_MAX_N 8

/* Lattice and domain.  2-D grids use NFE_D2Q9 with nz = 1.  A set bit of
 * wall_mask puts halfway walls at -1/2 and n_axis - 1/2 on that axis
 * (Sec. III C); the other axes are periodic. */
typedef struct {
    int lattice;              /* NFE_D2Q9 or NFE_D3Q19 */
    int nx, ny, nz;           /* nodes per axis, each >= 1 (nz = 1 for D2Q9); nx*ny*nz < 2^31 */
    unsigned wall_mask;       /* NFE_WALL_* bits; NFE_WALL_Z is invalid for D2Q9 */
} nfe_grid;

/* Device memory hooks (nfe_params.device_alloc / device_free), e.g. a framework's caching
 * allocator.  alloc returns device memory of at least `bytes` on the current GPU, aligned to
 * 256 bytes, or NULL (the call then fails with NFE_ENOMEM); free releases a pointer that alloc
 * returned.  Both are called on the thread that makes the library call. */
typedef void *(*nfe_alloc_fn)(size_t bytes, void *ctx);
typedef void (*nfe_free_fn)(void *ptr, void *ctx);

/* Physical and numerical parameters (Sec. II and Sec. III). */
typedef struct {
    const double *sigma;      /* N x N surface tensions, row-major, symmetric,
                                 zero diagonal, positive off-diagonal (host) */
    const double *tau;        /* N relaxation times tau_i > 1/2; omega+ = 1/tau of
                                 the component with the largest C (Eq. 42) (host) */
    double lambda_trt;        /* magic parameter of Eq. 26; < 0 selects BGK (omega- = omega+) */
    double m;                 /* coefficient m of g^eq (Eq. 40); mobility M = m (tau_g - 1/2) / 3 (Eq. 43) */
    double D;                 /* interface width (Sec. II; the paper uses 4) */
    double omega_stab;        /* Omega of Eq. 17; NaN selects 0 when every spreading
                                 parameter (Eq. 16) is negative and 1/90 otherwise */
    double body_force[3];     /* F_b (Eq. 2), lattice units */
    int precision;            /* NFE_FP64, NFE_FP32, NFE_FP32_F16STORE, NFE_FP32_BF16STORE */
    int implicit_component;   /* 0 .. N-1: the component computed as 1 - sum of the others */
    int flags;                /* NFE_NONCONSERVATIVE_FORCE | NFE_NO_PHI (ablations) */
    int scale_exp;            /* FP16 storage scale 2^scale_exp; ignored otherwise */
    void *cuda_stream;        /* cudaStream_t to queue work on (borrowed); NULL = default */
    double tau_g;             /* relaxation time of the component populations g (Sec. III B); 0 or 1
                                 selects tau_g = 1, where g* = g^eq and g needs no storage.  Other
                                 values (> 1/2) store the N-1 evolved components' g populations
                                 ((N-1) x Q planes, two buffers, compute type).  D3Q19: the split
                                 form of the step; batches: per-step launches on 32 x 8 tiles.
                                 NFE_EUNSUPPORTED with a geometry and together with NFE_NO_PHI */
    double component_force[3];    /* a body force acting on one component in proportion to its
                                     volume fraction, F += C_c F_c (the PaLS study of Sec. V drives
                                     only the droplet of fluid 2); all zero = none */
    int component_force_index;    /* c, 0 .. N-1 (user order; ignored when the force is zero) */
    nfe_alloc_fn device_alloc;    /* state, diagnostics and geometry buffers of the simulation come
                                     from here (both NULL: cudaMalloc / cudaFree).  Buffers are
                                     taken at nfe_create, at the first diagnostics call and at
                                     nfe_set_geometry, and given back at nfe_destroy (after the
                                     stream is synchronised) or when replaced.  The cuFFT plan of
                                     nfe_domain_size and a batch's own descriptors use cudaMalloc. */
    nfe_free_fn device_free;      /* set both or neither (NFE_EINVAL otherwise) */
    void *alloc_ctx;              /* passed through to both */
} nfe_params;

/* Global quantities of the current state, reduced on the GPU in FP64. */
typedef struct {
    int64_t step;                    /* time steps taken since create / set_fields */
    int N;
    double mass[NFE_MAX_N];          /* sum over sites of C_i */
    double momentum[3];              /* sum over sites of rho v, v of Eq. 37 (incl. F/2) */
    double force_sum[3];             /* sum over sites of F_s */
    double force_abs_sum[3];         /* sum over sites of |F_s| per axis */
    double max_abs_C[NFE_MAX_N];     /* max over sites of |C_i| */
    double min_C[NFE_MAX_N];         /* min over sites of C_i */
    double max_speed;                /* max over sites of |v| */
    int nonfinite;                   /* 1 if any population or volume fraction is NaN/Inf */
} nfe_diag;

/* Facts about a created simulation. */
typedef struct {
    int lattice, N, precision;
    int64_t sites;                   /* nx * ny * nz */
    double omega_stab;               /* Omega actually used */
    double factor_residual;          /* largest dropped coefficient of the factored flux
                                        potential, relative (checks alpha/Lambda/Theta) */
    int kernels_per_step;            /* kernel launches of one nfe_step(1) */
    int variant;                     /* tile shape in use (-1: not tuned yet) */
    int nvariants;                   /* tile shapes available for this lattice/N/precision */
    double min_bytes_per_site;       /* f (Q-1) and C (N-1) read once and written once (+ stored g, + the node class byte of a geometry) */
    size_t state_bytes;              /* size of the raw state (nfe_get_state) */
    size_t device_bytes;             /* device memory held by the simulation */
} nfe_info;

typedef struct nfe_sim nfe_sim;

/* Validate the arguments, build the tables of Sec. II (alpha and gamma from
 * Eqs. 8-9, Lambda from Eqs. 14-15, Theta from Eqs. 18-19, and the factored
 * flux potential S_i = C_i q_i(C) + (3D/4) lap C_i), allocate the device
 * state and set f = 0 (P = 0, v = 0) and C = 0.
 * Errors: NFE_EINVAL (bad grid, N outside 2..8, tau <= 1/2, sigma not
 * symmetric or not positive, bad precision or flags), NFE_ESINGULAR,
 * NFE_ENOMEM, NFE_ECUDA.  *out is NULL on error. */
nfe_status nfe_create(const nfe_grid *grid, int N, const nfe_params *params, nfe_sim **out);

/* Set the volume fractions (host, FP64, N x n; the row of the implicit
 * component is ignored and recomputed) and optionally the velocity (host,
 * FP64, 3 x n, or NULL for rest).  Populations are set to f^eq(P = 0, v)
 * (Eq. 27).  Resets the step counter.  Synchronises the stream. */
nfe_status nfe_set_fields(nfe_sim *sim, const double *C, const double *v);

/* Queue nsteps >= 0 time steps on the stream (asynchronous; replays a
 * captured CUDA graph).  Returns launch errors only; use nfe_sync or
 * nfe_diagnostics to learn about NFE_ENONFINITE. */
nfe_status nfe_step(nfe_sim *sim, int64_t nsteps);

/* Wait for the stream; NFE_ENONFINITE if a volume fraction went NaN/Inf. */
nfe_status nfe_sync(nfe_sim *sim);

/* Copy the current fields to host FP64 buffers (each may be NULL):
 * C (N x n, all components), v (3 x n, Eq. 37), P (n, Eq. 38).
 * Synchronises the stream. */
nfe_status nfe_fields(nfe_sim *sim, double *C, double *v, double *P);

/* Copy the populations f_k, k = 1 .. Q-1, to a host FP64 buffer ((Q-1) x n),
 * in the velocity order of Eqs. 20-21 (D2Q9) or, for D3Q19, +x, -x, +y, -y, +z, -z,
 * then the xy, xz and yz diagonals, each as (+,+), (-,-), (+,-), (-,+) (the opposite of
 * an odd k is k + 1).  f_0 is not kept: it feeds no moment.  Synchronises. */
nfe_status nfe_populations(nfe_sim *sim, double *f);

/* FP64 reductions of the current state on the GPU.  Synchronises. */
nfe_status nfe_diagnostics(nfe_sim *sim, nfe_diag *out);

/* Domain size of the phase-separation study (Sec. IV, the equation for L_i):
 * lambda_i = H(C_i - 1/2) (H(0) = 1), its discrete Fourier transform over the grid
 * taken as periodic (cuFFT), and L_i = 2 pi sum_{k != 0} |lambda_i(k)|^2 /
 * sum_{k != 0} |k| |lambda_i(k)|^2 with k = 2 pi (m_x / n_x, m_y / n_y, m_z / n_z),
 * the folded integer m in (-n/2, n/2].
 * L: host, N + 1 doubles: L_i in the user's component order, then their mean over
 *    the finite ones (a component without interface, lambda uniform, gives NaN).
 * nbins > 0: also the circularly averaged S_c(k) = <|lambda_c(k)|^2> of user
 *    component `component` in shells |k| ~ b dk, b = 1 .. nbins, dk = 2 pi / min(n_x,
 *    n_y[, n_z]) (host, nbins doubles; 0 for an empty shell).  nbins = 0: Sk unused.
 * The cuFFT plan and scratch are allocated on the first call and kept with the
 * simulation.  NFE_EINVAL for NULL L, nbins outside 0..2^20 or, with nbins > 0,
 * NULL Sk or a component outside 0..N-1.  Synchronises. */
nfe_status nfe_domain_size(nfe_sim *sim, double *L, int component, int nbins, double *Sk);

/* Open and complex boundaries (Sec. III C, the conditions that the emulsion and
 * patterned-surface applications of Sec. V use), on D2Q9 and D3Q19: solid nodes, inlets and the
 * convective outflow.
 * node: host, n bytes, one class per site (x fastest): 0 fluid, 1 solid, 2 + j inlet j;
 *   NULL removes the geometry (ninlets, inlets and outflow are then ignored).
 * inlets: host, ninlets x (D + N) doubles (D = 2 on D2Q9, 3 on D3Q19), row j = v_b (x, y,
 *   and z on D3Q19) then C_b of all N components in the user's order (finite, >= 0, summing
 *   to 1 within 1e-9);
 *   0 <= ninlets <= 64, NULL when ninlets = 0.
 * outflow: nonzero = convective outflow on the x = nx - 1 edge (a column on D2Q9, a plane on
 *   D3Q19); then column (plane) 0 must hold no fluid node, column nx - 1 no inlet node,
 *   nx >= 3 and the x axis no wall.  Column below means every (y, z) line's site x.
 * Rules: a solid node takes halfway bounce-back for f and for the component
 *   populations, and a neighbour inside it takes the value at x in every directional
 *   difference; links from inlet j carry f_k(x, t+1) = f*_kbar(x) + 2 w_k (e_k . v_b) /
 *   c_s^2 (e_k the entering direction, rho_b = 1) and the component equilibrium
 *   g^eq_k(C_b, v_b, S_b) of the prescribed state (S_b: Eq. 12 at the uniform C_b), and
 *   directional differences see C_b there; the outflow replaces every population and
 *   volume fraction of a fluid node in column nx - 1 by (old + U new(x - 1)) / (1 + U),
 *   U the mean x-momentum of the fluid nodes of column nx - 2 after streaming, and keeps a
 *   ghost column of volume fractions (convected the same way, started from column nx - 1)
 *   for the directional differences of column nx - 1.  Non-fluid nodes keep their
 *   populations and volume fractions; C := C_b on the inlet nodes now and at every
 *   nfe_set_fields.  nfe_fields reports v = P = F_s = 0 on solid nodes and v = v_b, P = 0 on
 *   inlet nodes.  With outflow the raw state (nfe_get_state) also holds the ghost column,
 *   so set the geometry before restoring a state.
 * Errors: NFE_EUNSUPPORTED for tau_g != 1 or NFE_NO_PHI;
 *   NFE_EINVAL for a class
 *   outside 0 .. 1 + ninlets, a bad inlet row or a violated outflow condition (these leave
 *   the previous geometry in place); NFE_ENOMEM or NFE_ECUDA while the new geometry is being
 *   uploaded, after which the simulation has no geometry (fully periodic / edge walls only)
 *   and the caller sets one again.
 * Synchronises the stream. */
nfe_status nfe_set_geometry(nfe_sim *sim, const uint8_t *node, int ninlets, const double *inlets, int outflow);

/* Raw state (checkpoint / resume, host buffer of info.state_bytes bytes):
 * populations and evolved volume fractions in device format, plus the step
 * counter (and, with an outflow, the ghost column).  get then set restores the
 * simulation bit for bit. */
nfe_status nfe_get_state(nfe_sim *sim, void *host_buf, size_t bytes);
nfe_status nfe_set_state(nfe_sim *sim, const void *host_buf, size_t bytes);

nfe_status nfe_get_info(const nfe_sim *sim, nfe_info *out);

/* Tile shape of the time-step kernel.  variant < 0 (the default) lets the
 * first nfe_step time every shape on the current state and keep the fastest
 * (the state is not modified); 0 .. nvariants-1 fixes one.  All shapes give
 * bit-identical results. */
nfe_status nfe_set_variant(nfe_sim *sim, int variant);

/* Kernel timing on the simulation's stream: when enabled, CUDA events bracket
 * every kernel launch of nfe_step (graphs are bypassed).  read returns, per
 * kernel kind, the launch count and total milliseconds since the last reset.
 * names[i] points to static strings. */
nfe_status nfe_profile_enable(nfe_sim *sim, int on);
nfe_status nfe_profile_read(nfe_sim *sim, int max_kinds, int *kinds,
                            const char **names, int64_t *launches, double *total_ms);

void nfe_destroy(nfe_sim *sim);

/* Host-only evaluation (no GPU) of the library's factored bulk flux potential
 * S_i = C_i q_i(C), i.e. sum_j alpha_ij (dE_B/dC_j + phi_j + xi_j) of Eq. 12
 * without its Laplacian terms, exactly as the kernels evaluate it, at npts
 * points C (host, npts x N, row-major, on the simplex).  S (host, npts x N)
 * receives S_i for the evolved components and 0 for the implicit one.  Same
 * validation and errors as nfe_create for sigma, D, omega_stab and
 * implicit_component. */
nfe_status nfe_bulk_potential_host(int N, const double *sigma, double D, double omega_stab,
                                   int implicit_component, int npts, const double *C, double *S);

const char *nfe_status_string(nfe_status s);
const char *nfe_last_error(void);

/* ---- Batched sweep of independent D2Q9 simulations (one persistent launch) ----
 * Many small simulations of different grid sizes and component counts (the
 * parameter sweeps of the lens and Janus benchmarks, Sec. IV A) advanced
 * together.  Every simulation is a full nfe_sim internally; nfe_batch_step
 * advances all of them by nsteps with ONE cooperative kernel launch (replayed
 * from a CUDA graph) whose CTAs walk the (simulation, tile) work list and meet
 * at a grid barrier between steps.  The barrier's wait is bounded: when it
 * runs out (NFE_ETIMEOUT from nfe_batch_sync) the kernel returns early and the
 * states are undefined, but the GPU context stays usable.
 * Constraints: D2Q9 grids, N = 2..5, one precision for the whole batch
 * (NFE_FP32 or NFE_FP64), params[i].cuda_stream ignored (params[0]'s is used).  Members with
 * NFE_NO_PHI or tau_g != 1 run in the per-step form on 32 x 8 tiles: with such a member,
 * nfe_batch_set_mode(NFE_BATCH_PERSISTENT) and nfe_batch_set_barrier_test return
 * NFE_EUNSUPPORTED. */
typedef struct nfe_batch nfe_batch;

typedef struct {
    int nsims;
    int64_t sites;                   /* total over all simulations */
    int nitems;                      /* (simulation, tile) work items per step */
    int grid;                        /* CTAs of the persistent launch */
    int tile_x, tile_y;              /* tile shape chosen by the autotuner (0 before the first step) */
    int graphs;                      /* 1 when launches are replayed from CUDA graphs */
    int form;                        /* launch form in use (NFE_BATCH_PERSISTENT or _PER_STEP), -1 before tuning */
} nfe_batch_info;

enum { NFE_BATCH_PERSISTENT = 0,   /* one cooperative launch for all nsteps */
       NFE_BATCH_PER_STEP = 1,     /* one batched launch per step (all captured in one graph) */
       NFE_BATCH_AUTO = 2 };       /* default: the autotuner times both forms and every tile
                                      shape at the first step and keeps the fastest */

/* grids, N and params are arrays of nsims entries (host).  Errors as nfe_create
 * for each simulation, plus NFE_EUNSUPPORTED for D3Q19 or N > 5. */
nfe_status nfe_batch_create(int nsims, const nfe_grid *grids, const int *N, const nfe_params *params,
                            nfe_batch **out);
/* As nfe_set_fields for simulation `sim` (0 .. nsims-1).  Resets its step counter. */
nfe_status nfe_batch_set_fields(nfe_batch *b, int sim, const double *C, const double *v);
/* Queue nsteps time steps of every simulation (asynchronous). */
nfe_status nfe_batch_step(nfe_batch *b, int64_t nsteps);
nfe_status nfe_batch_set_mode(nfe_batch *b, int mode);
/* Wait; NFE_ETIMEOUT if a barrier wait ran out, NFE_ENONFINITE if a volume fraction
 * of any simulation became NaN/Inf. */
nfe_status nfe_batch_sync(nfe_batch *b);
/* As nfe_fields / nfe_diagnostics for simulation `sim`.  Synchronise. */
nfe_status nfe_batch_fields(nfe_batch *b, int sim, double *C, double *v, double *P);
nfe_status nfe_batch_diagnostics(nfe_batch *b, int sim, nfe_diag *out);
nfe_status nfe_batch_get_info(const nfe_batch *b, nfe_batch_info *out);
/* Fault-injection hook for tests of the timeout path: the next launch (persistent form)
 * uses at most `spins` polls per barrier wait and its barriers wait for
 * `extra` more CTAs than the grid has (extra > 0 makes every wait run out).
 * spins <= 0 restores the default limit (about a second or more). */
nfe_status nfe_batch_set_barrier_test(nfe_batch *b, int64_t spins, int extra);
void nfe_batch_destroy(nfe_batch *b);

/* Allocation-free FP64 statistics of device-resident fields.  The paper has no
 * counterpart: this is a service for callers that cannot call cudaMalloc, such
 * as code running inside another runtime's memory pool or a fixed arena, where
 * an extra device allocation would fail or escape the owner's accounting.
 *
 * d_planes: device, nplanes x n doubles, plane p at d_planes[p * n] (for
 * example the C, v or P arrays of nfe_fields copied to the device).  d_out:
 * device, 4 x nplanes doubles; for plane p it receives the sum, the sum of
 * absolute values, the largest absolute value and the smallest value, at
 * d_out[4 p + 0 .. 3].  Work is queued on cuda_stream (NULL = legacy default
 * stream) and the call returns without waiting.
 *
 * It allocates nothing: the per-block partial sums live in one static device
 * array of the library (512 blocks x NFE_STATS_MAX_PLANES planes x 4 doubles,
 * 256 KiB), held by every GPU that loads the library until the process
 * exits.  Every call writes all the partials it later reads, so nothing has
 * to start at zero, but all calls share that array: calls whose work overlaps
 * on one GPU (for example calls queued on two different streams) race and
 * may return wrong results.  Each GPU has its own copy of the array.  The
 * first call on each device
 * looks up the array's device address with that device current; make that
 * first call before any stream capture.
 * A plane holding a NaN reports NaN as its sums, its largest absolute value
 * and its smallest value.
 * Errors: NFE_EINVAL when nplanes is outside 1..NFE_STATS_MAX_PLANES, n is
 * outside 1..2^40 or a pointer is NULL (nothing is launched); NFE_ECUDA when
 * the address lookup or a launch fails.  The message is in nfe_last_error(). */
#define NFE_STATS_MAX_PLANES 16
nfe_status nfe_field_stats_static(int nplanes, int64_t n, const double *d_planes, double *d_out,
                                  void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* NFE_H */
