// Internal interface of the domain-size diagnostic (nfe_spectrum.cu).
#pragma once

#include <string>

#include "nfe_internal.h"

namespace nfe {

struct Spectrum;   // cuFFT plan and scratch of one simulation

nfe_status spectrum_create(const Geom &g, int N, Spectrum **out, std::string &err);
void spectrum_destroy(Spectrum *sp);

// L (N + 1 host values: L_i in user order, then their mean over the finite ones) and, when
// nbins > 0, the shell-averaged S(k) of `component` (host, nbins values), from the FP64 C
// planes of all N components in user order (device).
nfe_status domain_size(Spectrum *sp, int N, const double *C, int component, int nbins, double *L, double *Sk,
                       cudaStream_t st, std::string &err);

}  // namespace nfe
