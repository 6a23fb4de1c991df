// Host-side Sec. II tables (see nfe_tables.cpp).
#pragma once

#include <string>
#include <vector>

#include "../../include/nfe.h"

namespace nfe {

struct Tables {
    int N = 0;
    double omega = 0.0;
    std::vector<double> beta, kappa, alpha, gamma;   // N x N (internal order), gamma N
    std::vector<double> q2;                           // (N-1) x N(N+1)/2, monomials a <= b
    std::vector<double> q4;                           // (N-1) x mono4s_count(N), structured quartic part (Omega != 0)
    std::vector<double> r3;                           // (N-1) x mono3r_count(N), cubic remainder without C_i (no phi)
    double residual = 0.0;                            // largest dropped coefficient, relative
    int lambda_count = 0;
};

// sigma_user: N x N in the user's order; uidx[a] = user index of internal slot a.
nfe_status build_tables(int N, const double *sigma_user, const int *uidx, double D, double omega,
                        bool with_phi, Tables &out, std::string &err);

// Whether any spreading parameter (Eq. 16) is non-negative.
bool auto_omega(int N, const double *sigma);

}  // namespace nfe
