// Internal interface of the batched persistent kernel (nfe_batch.cu) and its host side.
#pragma once

#include <stddef.h>

#include "nfe_internal.h"

#define NFE_BATCH_ERR_TIMEOUT 1

namespace nfe {

constexpr int kBatchMaxN = 5;   // component counts 2..5 in a batch
// forms of a batch member's step: 0 the method as stated, 1 the no-phi ablation (flux potential
// without phi_j), 2 stored component populations (tau_g != 1)
constexpr int kBatchForms = 3;
constexpr int kBatchGroups = (kBatchMaxN - 1) * kBatchForms;   // work-list group (N - 2) * kBatchForms + form

// One simulation as the batched kernel sees it (device memory, read-only).
// The coefficients come last: the kernel copies the descriptor into shared memory
// up to (not including) Coef::q4c, since it reads the degree-4 table from device memory.
template <typename T>
struct __align__(16) BatchSim {
    Geom geom;
    int N;
    int form;               // 0, 1 or 2, as kBatchForms above
    void *f[2];
    void *C[2];
    void *g[2];             // component populations (form 2), else null
    int *flag;
    Coef<T> coef;
};

// Grid-barrier state (device memory): arrival count, generation, work-item ticket, error word.
// Every launch resets the words before `error` (kBatchSyncResetBytes); the error word is sticky:
// a barrier timeout stays recorded through later launches (whose barriers then release at once,
// so they do no work) until nfe_batch_sync reports and clears it.
struct BatchSync {
    unsigned count;
    unsigned generation;
    unsigned long long ticket;   // work-item counter of the persistent kernel
    int error;
    int pad_;
};
constexpr size_t kBatchSyncResetBytes = offsetof(BatchSync, error);

struct BatchLaunch {
    const void *sims;       // BatchSim<T>[nsims]
    const int4 *items;      // (sim, x0, y0, 0) work items
    int nitems;
    int nsteps;
    int parity;             // buffer holding the current state of every simulation
    BatchSync *sync;
    long long spin_limit;   // polls before a barrier wait gives up
    unsigned expected;      // CTAs a barrier waits for (normally the grid size)
    int grid;
    int nstart[kBatchGroups];     // items of group q (N = 2 + q / kBatchForms, form q % kBatchForms):
    int ncount[kBatchGroups];     // [nstart[q], nstart[q] + ncount[q])
};

using BatchSetup = cudaError_t (*)(int *blocks_per_sm);
using BatchLauncher = cudaError_t (*)(const BatchLaunch &, cudaStream_t);

constexpr int kBatchVariants = 2;
struct BatchOps {
    int ty[kBatchVariants];                     // tile heights (TX = 32)
    BatchSetup setup[kBatchVariants];
    BatchLauncher persistent[kBatchVariants];   // one cooperative launch for all steps
    BatchLauncher per_step[kBatchVariants];     // one launch per step
};

const BatchOps *batch_ops(int prec);

}  // namespace nfe
