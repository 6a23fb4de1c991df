// Batched sweep: many independent D2Q9 simulations (mixed grid sizes and
// component counts) advanced by ONE persistent kernel launch for many time
// steps.  Each CTA walks a static share of the (simulation, tile) work list,
// running the fused tile step of nfe_fused2d.cuh with that simulation's
// coefficients (read from global memory), and all CTAs meet at a grid barrier
// between time steps.  The launch is cooperative (all CTAs co-resident), and
// the barrier's wait is bounded: after `spin_limit` polls a CTA records a
// timeout in the error word and every CTA leaves the step loop, so a fault in
// the barrier can never hang the GPU.
#include <cuda_runtime.h>

#include <cstddef>

#include "nfe_batch.h"
#include "nfe_fused2d.cuh"

namespace nfe {

// Returns false when the barrier timed out (or another CTA reported an error).
__device__ __forceinline__ bool grid_barrier(BatchSync *sync, unsigned nblocks, long long spin_limit) {
    // nblocks: arrivals that release the barrier (the grid size; larger in the timeout test)
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &sync->generation;
        volatile int *err = &sync->error;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(&sync->count, 1u) + 1u;
        if (arrived == nblocks) {
            sync->count = 0u;
            __threadfence();
            atomicAdd(&sync->generation, 1u);
        } else {
            long long spins = 0;
            while (*gen == g && *err == 0) {
                if (++spins > spin_limit) { atomicExch(&sync->error, NFE_BATCH_ERR_TIMEOUT); break; }
                __nanosleep(100);
            }
        }
        __threadfence();
        ok = (*err == 0);
    }
    __syncthreads();
    return ok != 0;
}

// The tile's simulation descriptor (geometry, coefficients, pointers) -> shared memory, up to
// the inline quartic table, which these kernels do not read (they read its device-memory copy:
// loop-invariant loads from the shared descriptor would be hoisted into registers and spill).
template <typename T>
__device__ __forceinline__ void load_desc(const BatchSim<T> &dg, BatchSim<T> &d) {
    static_assert(sizeof(BatchSim<T>) % 16 == 0, "16-byte copies");
    constexpr size_t used = offsetof(BatchSim<T>, coef) + offsetof(Coef<T>, q4c);
    constexpr int n16 = int((used + 15) / 16);
    static_assert(n16 * 16 <= sizeof(BatchSim<T>), "copy inside the descriptor");
    const int4 *src = reinterpret_cast<const int4 *>(&dg);
    int4 *dst = reinterpret_cast<int4 *>(&d);
    for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
}

template <typename T, typename SF, int TX, int TY, int NN, bool L2ONLY>
__device__ __forceinline__ void batch_tile_n(const BatchSim<T> &d, int cur, int x0, int y0, unsigned char *smem) {
    fused2d_tile<NN, T, SF, TX, TY, L2ONLY, Q4_GLOBAL>(d.geom, d.coef, static_cast<const SF *>(d.f[cur]),
                                                      static_cast<SF *>(d.f[1 - cur]), static_cast<const T *>(d.C[cur]),
                                                      static_cast<T *>(d.C[1 - cur]), d.flag, x0, y0, smem);
}

// Any N (2..5) in one non-inlined function: the persistent form, whose CTAs meet simulations of
// every N.  L2-only loads: inside one launch, other CTAs' writes of the previous step must not
// be read from a stale L1 line.
template <typename T, typename SF, int TX, int TY>
__device__ __noinline__ void batch_tile(const BatchSim<T> &dg, int cur, int x0, int y0, unsigned char *smem) {
    __shared__ __align__(16) BatchSim<T> d;
    load_desc(dg, d);
    __syncthreads();
    switch (d.N) {
        case 2: batch_tile_n<T, SF, TX, TY, 2, true>(d, cur, x0, y0, smem); break;
        case 3: batch_tile_n<T, SF, TX, TY, 3, true>(d, cur, x0, y0, smem); break;
        case 4: batch_tile_n<T, SF, TX, TY, 4, true>(d, cur, x0, y0, smem); break;
        default: batch_tile_n<T, SF, TX, TY, 5, true>(d, cur, x0, y0, smem); break;
    }
}

// registers per thread are bounded so that several CTAs share an SM
template <typename T, int NT> struct BatchOcc { static constexpr int value = sizeof(T) == 4 ? (NT <= 128 ? 6 : 3) : (NT <= 128 ? 4 : 2); };

// the persistent kernel keeps its loop state live across the (non-inlined) tile
// call, so it gets a larger register budget than the one-launch-per-step form
template <typename T, int NT> struct PersistOcc { static constexpr int value = sizeof(T) == 4 ? (NT <= 128 ? 4 : 2) : (NT <= 128 ? 3 : 1); };

template <typename T, typename SF, int TX, int TY>
__global__ void __launch_bounds__(TX * TY, (PersistOcc<T, TX * TY>::value))
k_batch_persistent(const BatchSim<T> *__restrict__ sims, const int4 *__restrict__ items, int nitems,
                   int nsteps, int parity0, BatchSync *sync, long long spin_limit, unsigned expected) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // Work is handed out dynamically by one counter that only grows: step t owns the
    // indices [t * nitems, (t + 1) * nitems).  A CTA that draws an index of the next
    // step keeps it and starts the next step with it.
    // The following index is drawn when a tile starts and read when it ends, so the atomic's
    // round trip overlaps the tile instead of stalling the CTA between tiles.
    __shared__ long long next;
    if (threadIdx.x == 0) next = (long long)atomicAdd(&sync->ticket, 1ull);
    __syncthreads();
    for (int t = 0; t < nsteps; ++t) {
        const int cur = (parity0 + t) & 1;
        const long long end = (long long)(t + 1) * nitems;
        long long idx = next;
        while (idx < end) {
            unsigned long long drawn = 0ull;
            if (threadIdx.x == 0) drawn = atomicAdd(&sync->ticket, 1ull);
            const int4 w = items[idx - (long long)t * nitems];
            batch_tile<T, SF, TX, TY>(sims[w.x], cur, w.y, w.z, smem_raw);
            __syncthreads();      // shared memory is reused by the next tile
            if (threadIdx.x == 0) next = (long long)drawn;
            __syncthreads();
            idx = next;
        }
        if (t + 1 < nsteps && !grid_barrier(sync, expected, spin_limit)) return;
    }
}

// One launch per step and per (component count, form), one CTA per work item (the
// non-persistent batched form).  The work list is grouped that way, so each launch covers one
// contiguous range and carries a single inlined tile body (smaller code, its own register
// allocation, no switch).  FORM 1: the no-phi flux potential; FORM 2: stored component
// populations (tau_g != 1; 32 x 8 tiles only).
template <typename T, typename SF, int TX, int TY, int NN, int FORM>
__global__ void __launch_bounds__(TX * TY, (BatchOcc<T, TX * TY>::value))
k_batch_step(const BatchSim<T> *__restrict__ sims, const int4 *__restrict__ items, int parity) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) BatchSim<T> d;
    const int4 w = items[blockIdx.x];
    const BatchSim<T> &dg = sims[w.x];
    // the coefficients go to shared memory while the tile's own loads are already in flight:
    // geometry and pointers are read straight from the descriptor (one broadcast load each),
    // and the tile waits for the copy only before its first use of the coefficients
    load_desc(dg, d);
    const Geom geom = dg.geom;
    constexpr int Q4 = FORM == 1 ? Q4_NOPHI : Q4_GLOBAL;
    fused2d_tile<NN, T, SF, TX, TY, false, Q4, FORM == 2, false, true>(
        geom, d.coef, static_cast<const SF *>(dg.f[parity]), static_cast<SF *>(dg.f[1 - parity]),
        static_cast<const T *>(dg.C[parity]), static_cast<T *>(dg.C[1 - parity]), dg.flag, w.y, w.z, smem_raw,
        FORM == 2 ? static_cast<const T *>(dg.g[parity]) : nullptr, FORM == 2 ? static_cast<T *>(dg.g[1 - parity]) : nullptr);
}

template <typename T, int TX, int TY>
constexpr size_t batch_smem() { return Fused2DShape<5, T, TX, TY>::BYTES; }

template <typename T, typename SF, int TX, int TY>
struct BatchKernels {
    // the stored-population form exists for 32 x 8 tiles only
    static constexpr bool kHasForm2 = TY == 8;
    template <int NN, int FORM>
    static cudaError_t step_attr() {
        if constexpr (FORM == 2 && !kHasForm2) {
            return cudaSuccess;
        } else {
            return cudaFuncSetAttribute(k_batch_step<T, SF, TX, TY, NN, FORM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        int(Fused2DShape<NN, T, TX, TY>::BYTES));
        }
    }
    template <int NN>
    static cudaError_t step_attr_n() {
        cudaError_t e = step_attr<NN, 0>();
        if (e == cudaSuccess) e = step_attr<NN, 1>();
        if (e == cudaSuccess) e = step_attr<NN, 2>();
        return e;
    }
    static cudaError_t setup(int *blocks_per_sm) {
        const size_t smem = batch_smem<T, TX, TY>();
        cudaError_t e = cudaFuncSetAttribute(k_batch_persistent<T, SF, TX, TY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
        if (e != cudaSuccess) return e;
        if ((e = step_attr_n<2>()) != cudaSuccess || (e = step_attr_n<3>()) != cudaSuccess ||
            (e = step_attr_n<4>()) != cudaSuccess || (e = step_attr_n<5>()) != cudaSuccess)
            return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_batch_persistent<T, SF, TX, TY>,
                                                             TX * TY, smem);
    }
    static cudaError_t persistent(const BatchLaunch &L, cudaStream_t st) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(L.grid);
        cfg.blockDim = dim3(TX * TY);
        cfg.dynamicSmemBytes = batch_smem<T, TX, TY>();
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, k_batch_persistent<T, SF, TX, TY>,
                                  static_cast<const BatchSim<T> *>(L.sims), L.items, L.nitems, L.nsteps,
                                  L.parity, L.sync, L.spin_limit, L.expected);
    }
    template <int NN, int FORM>
    static void step_nf(const BatchLaunch &L, int parity, cudaStream_t st) {
        const int q = (NN - 2) * kBatchForms + FORM;
        if (L.ncount[q] <= 0) return;
        if constexpr (FORM == 2 && !kHasForm2) {
            return;                       // never listed: the host keeps such batches on 32 x 8 tiles
        } else {
            k_batch_step<T, SF, TX, TY, NN, FORM><<<L.ncount[q], TX * TY, Fused2DShape<NN, T, TX, TY>::BYTES, st>>>(
                static_cast<const BatchSim<T> *>(L.sims), L.items + L.nstart[q], parity);
        }
    }
    template <int NN>
    static void step_n(const BatchLaunch &L, int parity, cudaStream_t st) {
        step_nf<NN, 0>(L, parity, st);
        step_nf<NN, 1>(L, parity, st);
        step_nf<NN, 2>(L, parity, st);
    }
    static cudaError_t per_step(const BatchLaunch &L, cudaStream_t st) {
        for (int t = 0; t < L.nsteps; ++t) {
            const int parity = (L.parity + t) & 1;
            step_n<2>(L, parity, st);
            step_n<3>(L, parity, st);
            step_n<4>(L, parity, st);
            step_n<5>(L, parity, st);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
};

template <typename T, typename SF>
const BatchOps *batch_ops_for() {
    static const BatchOps o = {
        {4, 8},
        {&BatchKernels<T, SF, 32, 4>::setup, &BatchKernels<T, SF, 32, 8>::setup},
        {&BatchKernels<T, SF, 32, 4>::persistent, &BatchKernels<T, SF, 32, 8>::persistent},
        {&BatchKernels<T, SF, 32, 4>::per_step, &BatchKernels<T, SF, 32, 8>::per_step},
    };
    return &o;
}

const BatchOps *batch_ops(int prec) {
    switch (prec) {
        case NFE_FP64: return batch_ops_for<double, double>();
        case NFE_FP32: return batch_ops_for<float, float>();
        default: return nullptr;
    }
}

}  // namespace nfe
