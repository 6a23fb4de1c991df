// Sec. II tables of arXiv 2605.22214, built once per simulation on the host in
// FP64: alpha and gamma (Eqs. 8-9), Lambda (Eqs. 14-15), Theta (Eqs. 18-19)
// and the coefficients of the factored flux potential
//   S_i = C_i q_i(C) + (3D/4) lap C_i   (equal to Eq. 12 on the simplex):
// the quadratic part of q_i as monomial coefficients, and the quartic (stabiliser,
// Eq. 17) part in the structured form
//   q4_i = C_i sum_{l != i} C_l^2 sum_{m not in {i,l}} a_{ilm} C_m
//        + sum_{k < l; i not in {k,l}} b_{ikl} C_k^2 C_l^2,
// which follows from xi_j = (12 Omega / D) sum_{k<l} C_k^2 C_l^2 inner_j^{kl}(C) with
// inner_j^{kl} linear: the pairs that contain i carry C_i^2, and for the others the
// Theta conditions (Eqs. 18-19) leave only the C_i term of sum_j alpha_ij inner_j^{kl}.
#include "nfe_tables.h"

#include "nfe_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <map>
#include <vector>

namespace nfe {

namespace {

// ---- dense linear algebra (Gauss-Jordan with partial pivoting) -------------

// Solves A X = B in place (A: n x n, B: n x r, row-major).  Returns false when
// a pivot falls below tol * max|A|.
bool gauss_solve(std::vector<double> A, int n, std::vector<double> &B, int r, double tol = 1e-13) {
    double amax = 0.0;
    for (double a : A) amax = std::max(amax, std::fabs(a));
    if (n == 0) return true;
    if (amax == 0.0) return false;
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int i = col + 1; i < n; ++i)
            if (std::fabs(A[i * n + col]) > std::fabs(A[piv * n + col])) piv = i;
        if (std::fabs(A[piv * n + col]) <= tol * amax) return false;
        if (piv != col) {
            for (int j = 0; j < n; ++j) std::swap(A[col * n + j], A[piv * n + j]);
            for (int j = 0; j < r; ++j) std::swap(B[col * r + j], B[piv * r + j]);
        }
        const double d = A[col * n + col];
        for (int j = 0; j < n; ++j) A[col * n + j] /= d;
        for (int j = 0; j < r; ++j) B[col * r + j] /= d;
        for (int i = 0; i < n; ++i) {
            if (i == col) continue;
            const double f = A[i * n + col];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) A[i * n + j] -= f * A[col * n + j];
            for (int j = 0; j < r; ++j) B[i * r + j] -= f * B[col * r + j];
        }
    }
    return true;
}

// ---- sparse polynomials over C_0..C_{N-1}, exponents packed 4 bits each ----

using Mono = uint32_t;
using Poly = std::map<Mono, double>;

Mono var_mono(int i) { return Mono(1) << (4 * i); }
int mono_exp(Mono m, int i) { return int((m >> (4 * i)) & 0xF); }
int mono_deg(Mono m) { int d = 0; for (int i = 0; i < 8; ++i) d += mono_exp(m, i); return d; }

void axpy(Poly &y, double a, const Poly &x) {
    if (a == 0.0) return;
    for (const auto &kv : x) y[kv.first] += a * kv.second;
}
Poly mul(const Poly &a, const Poly &b) {
    Poly out;
    for (const auto &x : a)
        for (const auto &y : b) out[x.first + y.first] += x.second * y.second;
    return out;
}
Poly var(int i) { return Poly{{var_mono(i), 1.0}}; }
Poly constant(double c) { return Poly{{Mono(0), c}}; }

// f'(L) - f'(L + K) with f'(u) = 2u - 6u^2 + 4u^3 (Eq. 7)
Poly fprime(const Poly &L) {
    Poly L2 = mul(L, L), L3 = mul(L2, L);
    Poly out;
    axpy(out, 2.0, L);
    axpy(out, -6.0, L2);
    axpy(out, 4.0, L3);
    return out;
}

double max_abs(const Poly &p) {
    double m = 0.0;
    for (const auto &kv : p) m = std::max(m, std::fabs(kv.second));
    return m;
}

}  // namespace

nfe_status build_tables(int N, const double *sigma_user, const int *uidx, double D, double omega,
                        bool with_phi, Tables &out, std::string &err) {
    out = Tables();
    out.N = N;
    out.omega = omega;
    // internal order: slot a holds user component uidx[a] (implicit one last)
    std::vector<double> s(N * N);
    for (int a = 0; a < N; ++a)
        for (int b = 0; b < N; ++b) s[a * N + b] = sigma_user[uidx[a] * N + uidx[b]];
    out.beta.assign(N * N, 0.0);
    out.kappa.assign(N * N, 0.0);
    for (int i = 0; i < N * N; ++i) {
        out.beta[i] = 6.0 * s[i] / D;       // D = sqrt(8 kappa / beta), sigma = sqrt(2 kappa beta / 9)
        out.kappa[i] = 0.75 * D * s[i];
    }

    // alpha = sigma^-1 - (sigma^-1 1)(1^T sigma^-1) / (1^T sigma^-1 1), gamma = -(sigma^-1 1) / (1^T sigma^-1 1):
    // the unique solution of alpha sigma = I + gamma 1^T, alpha 1 = 0 (Eqs. 8-9) when sigma is invertible.
    std::vector<double> inv(N * N, 0.0);
    for (int i = 0; i < N; ++i) inv[i * N + i] = 1.0;
    if (!gauss_solve(s, N, inv, N)) { err = "surface-tension matrix is singular (Eqs. 8-9)"; return NFE_ESINGULAR; }
    std::vector<double> u(N, 0.0);
    double tot = 0.0;
    for (int i = 0; i < N; ++i) { for (int j = 0; j < N; ++j) u[i] += inv[i * N + j]; tot += u[i]; }
    if (std::fabs(tot) < 1e-300) { err = "alpha/gamma system is singular (1^T sigma^-1 1 = 0)"; return NFE_ESINGULAR; }
    out.alpha.assign(N * N, 0.0);
    out.gamma.assign(N, 0.0);
    for (int i = 0; i < N; ++i) {
        out.gamma[i] = -u[i] / tot;
        for (int j = 0; j < N; ++j) out.alpha[i * N + j] = inv[i * N + j] - u[i] * u[j] / tot;
    }
    const auto A = [&](int i, int j) { return out.alpha[i * N + j]; };
    const auto S = [&](int i, int j) { return s[i * N + j]; };

    // Lambda_{j; jklm} for every triple k < l < m: sub-matrix of alpha over the
    // other N - 3 components times Lambda = Gamma (Eqs. 14-15).
    std::vector<Poly> phi(N);
    for (int k = 0; k < N; ++k)
        for (int l = k + 1; l < N; ++l)
            for (int m = l + 1; m < N; ++m) {
                std::vector<int> R;
                for (int j = 0; j < N; ++j) if (j != k && j != l && j != m) R.push_back(j);
                const int r = int(R.size());
                if (r == 0) continue;
                std::vector<double> M(r * r), rhs(r);
                for (int a = 0; a < r; ++a) {
                    const int i = R[a];
                    for (int b = 0; b < r; ++b) M[a * r + b] = A(i, R[b]);
                    rhs[a] = -6.0 * (A(i, k) * (S(k, l) + S(k, m)) + A(i, l) * (S(k, l) + S(l, m))
                                     + A(i, m) * (S(k, m) + S(l, m)) - out.gamma[i]);
                }
                if (!gauss_solve(M, r, rhs, 1)) { err = "alpha sub-matrix of a Lambda system is singular"; return NFE_ESINGULAR; }
                const Poly ckl = mul(mul(var(k), var(l)), var(m));
                for (int b = 0; b < r; ++b) {
                    if (with_phi) axpy(phi[R[b]], 12.0 / D * rhs[b], ckl);
                    out.lambda_count++;
                }
            }

    // Stabiliser part (Eq. 17) with Theta_{kl; j; m} from sub-matrix * Theta = 2 alpha_{., m}
    // (Eqs. 18-19), directly in the structured form above (layout per evolved i: the a_{ilm}
    // for l != i ascending and m ascending, then the b_{ikl} for k < l ascending).
    const int m4 = mono4s_count(N);
    out.q4.assign(omega != 0.0 ? (N - 1) * m4 : 0, 0.0);
    std::vector<double> q4max(N, 0.0), q4drop(N, 0.0);
    if (omega != 0.0) {
        const auto pos_a = [&](int i, int l, int m) {
            const int li = l - (l > i ? 1 : 0);
            const int mi = m - (m > i ? 1 : 0) - (m > l ? 1 : 0);
            return li * (N - 2) + mi;
        };
        const auto pos_b = [&](int i, int k, int l) {
            int r = (N - 1) * (N - 2);
            for (int a = 0; a < N; ++a)
                for (int b = a + 1; b < N; ++b) {
                    if (a == i || b == i) continue;
                    if (a == k && b == l) return r;
                    ++r;
                }
            return -1;
        };
        const double scale = 12.0 / D * omega;
        for (int k = 0; k < N; ++k)
            for (int l = k + 1; l < N; ++l) {
                // inner_j = 2 C_j - sum_m Theta_{kl;j;m} C_m for every j outside {k, l}
                std::vector<Poly> inner(N);
                for (int j = 0; j < N; ++j) if (j != k && j != l) inner[j] = mul(constant(2.0), var(j));
                for (int m = 0; m < N; ++m) {
                    if (m == k || m == l) continue;
                    std::vector<int> R;
                    for (int j = 0; j < N; ++j) if (j != k && j != l && j != m) R.push_back(j);
                    const int r = int(R.size());
                    if (r == 0) continue;
                    std::vector<double> M(r * r), rhs(r);
                    for (int a = 0; a < r; ++a) {
                        for (int b = 0; b < r; ++b) M[a * r + b] = A(R[a], R[b]);
                        rhs[a] = 2.0 * A(R[a], m);
                    }
                    if (!gauss_solve(M, r, rhs, 1)) { err = "alpha sub-matrix of a Theta system is singular"; return NFE_ESINGULAR; }
                    for (int b = 0; b < r; ++b) axpy(inner[R[b]], -rhs[b], var(m));
                }
                // G_i^{kl} = sum_j alpha_ij inner_j^{kl}, linear in C_m (m outside {k, l})
                for (int i = 0; i < N - 1; ++i) {
                    Poly G;
                    for (int j = 0; j < N; ++j) if (j != k && j != l) axpy(G, A(i, j), inner[j]);
                    const auto coef = [&](int m) { const auto it = G.find(var_mono(m)); return it == G.end() ? 0.0 : it->second; };
                    for (int m = 0; m < N; ++m) q4max[i] = std::max(q4max[i], std::fabs(scale * coef(m)));
                    if (i == k || i == l) {
                        const int o = i == k ? l : k;
                        for (int m = 0; m < N; ++m)
                            if (m != k && m != l) out.q4[i * m4 + pos_a(i, o, m)] = scale * coef(m);
                    } else {
                        out.q4[i * m4 + pos_b(i, k, l)] = scale * coef(i);
                        for (int m = 0; m < N; ++m)            // must vanish: divisibility by C_i
                            if (m != i) q4drop[i] = std::max(q4drop[i], std::fabs(scale * coef(m)));
                    }
                }
            }
    }

    // bulk chemical potential dE_B/dC_j (Eq. 7) as polynomials
    std::vector<Poly> mub(N);
    for (int j = 0; j < N; ++j) {
        const Poly fj = fprime(var(j));
        for (int k = 0; k < N; ++k) {
            if (k == j) continue;
            Poly sum = var(j);
            axpy(sum, 1.0, var(k));
            Poly d = fj;
            axpy(d, -1.0, fprime(sum));
            axpy(mub[j], out.beta[j * N + k], d);
        }
    }
    Poly ssum;
    for (int i = 0; i < N; ++i) axpy(ssum, 1.0, var(i));
    const Poly ssum2 = mul(ssum, ssum);

    // enumeration orders used by the kernels
    std::vector<Mono> mono2;
    for (int a = 0; a < N; ++a)
        for (int b = a; b < N; ++b) mono2.push_back(var_mono(a) + var_mono(b));

    out.q2.assign((N - 1) * mono2.size(), 0.0);
    // without phi_j the cubic keeps monomials free of C_i: kept as a remainder r_i(C), in the
    // order a <= b <= c over the components other than i
    const int m3 = mono3r_count(N);
    if (!with_phi) out.r3.assign((N - 1) * m3, 0.0);
    out.residual = 0.0;
    for (int i = 0; i < N - 1; ++i) {
        Poly cubic;
        for (int j = 0; j < N; ++j) {
            axpy(cubic, A(i, j), mub[j]);
            axpy(cubic, A(i, j), phi[j]);
        }
        // homogenise to degree 3 with powers of sum_k C_k (= 1 on the simplex)
        Poly h;
        for (const auto &kv : cubic) {
            const int d = mono_deg(kv.first);
            const Poly t{{kv.first, kv.second}};
            if (d == 3) axpy(h, 1.0, t);
            else if (d == 2) axpy(h, 1.0, mul(t, ssum));
            else if (d == 1) axpy(h, 1.0, mul(t, ssum2));
            else if (kv.second != 0.0) { err = "unexpected constant term in the flux potential"; return NFE_ESINGULAR; }
        }
        const double scale = std::max(max_abs(h), 1e-300);
        double rest = 0.0;
        std::vector<Mono> mono3r;
        for (int a = 0; a < N; ++a)
            for (int b = a; b < N; ++b)
                for (int c = b; c < N; ++c)
                    if (a != i && b != i && c != i) mono3r.push_back(var_mono(a) + var_mono(b) + var_mono(c));
        for (const auto &kv : h) {
            if (mono_exp(kv.first, i) == 0) {
                rest = std::max(rest, std::fabs(kv.second));
                if (!with_phi) {
                    const auto it = std::find(mono3r.begin(), mono3r.end(), kv.first);
                    out.r3[i * m3 + (it - mono3r.begin())] += kv.second;
                }
                continue;
            }
            const Mono q = kv.first - var_mono(i);
            const auto it = std::find(mono2.begin(), mono2.end(), q);
            out.q2[i * mono2.size() + (it - mono2.begin())] += kv.second;
        }
        out.residual = std::max(out.residual, rest / scale);
    }
    for (int i = 0; i < N - 1; ++i)
        if (q4max[i] > 0.0) out.residual = std::max(out.residual, q4drop[i] / q4max[i]);
    if (with_phi && out.residual > 1e-10) {
        err = "flux potential does not factor by C_i (Lambda/Theta solve inaccurate)";
        return NFE_ESINGULAR;
    }
    return NFE_OK;
}

bool auto_omega(int N, const double *sigma) {
    // true when some spreading parameter S_ij;k = sigma_ij - sigma_ik - sigma_jk (Eq. 16) is >= 0
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k) {
                if (i == j || j == k || i == k) continue;
                if (sigma[i * N + j] - sigma[i * N + k] - sigma[j * N + k] >= 0.0) return true;
            }
    return false;
}

}  // namespace nfe
