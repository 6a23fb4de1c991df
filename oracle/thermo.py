"""Sec. II of the paper: free energy, chemical potentials and the corrected flux.

Oracle code (test infrastructure only).  Components are indexed 0 .. N-1
here; the paper counts 1 .. N.  All arithmetic is float64.

Readings taken where the paper leaves a choice:
  * beta_ij = 6 sigma_ij / D and kappa_ij = 3 D sigma_ij / 4, the unique
    solution of D = sqrt(8 kappa / beta) and sigma = sqrt(2 kappa beta / 9)
    (Sec. II, after Eq. 5).
  * Sums over i != j in Eq. 5 run over ordered pairs, so every unordered pair
    enters E_B once with weight beta_ij and mu_j (Eq. 7) once per partner.
  * Omega (Eq. 17): the paper fixes Omega = 0 when every spreading parameter
    (Eq. 16) is negative and uses 1/90 or 1/18 otherwise; `default_omega`
    returns 0 or 1/90 accordingly when the caller passes NaN.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from .poly import Poly


class SingularSystem(ValueError):
    """An alpha/gamma, Lambda or Theta system had no unique solution."""


# ----------------------------------------------------------------------------
# Free-energy coefficients and the double-well f (Sec. II, Eq. 5 and Eq. 7)
# ----------------------------------------------------------------------------

def beta_kappa(sigma, D):
    """beta_ij = 6 sigma_ij / D, kappa_ij = 3 D sigma_ij / 4 (Sec. II, below Eq. 5)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    return 6.0 * sigma / D, 0.75 * D * sigma


def f_well(c):
    """f(C) = C^2 (1 - C)^2 (Eq. 5)."""
    return c * c * (1.0 - c) ** 2


def f_well_prime(c):
    """f'(C) = 2 C (1 - 3 C + 2 C^2) (Eq. 7)."""
    return 2.0 * c * (1.0 - 3.0 * c + 2.0 * c * c)


def bulk_energy(C, beta):
    """E_B = sum_{i != j} beta_ij / 2 [f(C_i) + f(C_j) - f(C_i + C_j)] (Eq. 5)."""
    N = C.shape[0]
    E = np.zeros(C.shape[1:])
    for i in range(N):
        for j in range(N):
            if i != j:
                E = E + 0.5 * beta[i, j] * (f_well(C[i]) + f_well(C[j]) - f_well(C[i] + C[j]))
    return E


def interface_energy(gradC, kappa):
    """E_I = -sum_{i != j} kappa_ij / 2 grad C_i . grad C_j (Eq. 5); gradC has shape (N, 3, ...)."""
    N = gradC.shape[0]
    E = np.zeros(gradC.shape[2:])
    for i in range(N):
        for j in range(N):
            if i != j:
                E = E - 0.5 * kappa[i, j] * np.sum(gradC[i] * gradC[j], axis=0)
    return E


# ----------------------------------------------------------------------------
# alpha / gamma (Eqs. 8-9), Lambda (Eqs. 14-15), Theta (Eqs. 18-19)
# ----------------------------------------------------------------------------

def alpha_gamma(sigma):
    """Solve alpha sigma = I + gamma 1^T together with alpha 1 = 0 (Eqs. 8-9).

    Unknowns: the N^2 entries of alpha (row-major) followed by the N entries
    of gamma.  Equation (i, j) of Eq. 8 reads sum_k alpha_ik sigma_kj - gamma_i
    = delta_ij; equation i of Eq. 9 reads sum_k alpha_ik = 0.
    """
    sigma = np.asarray(sigma, dtype=np.float64)
    N = sigma.shape[0]
    n_unk = N * N + N
    A = np.zeros((n_unk, n_unk))
    b = np.zeros(n_unk)
    row = 0
    for i in range(N):
        for j in range(N):
            for k in range(N):
                A[row, i * N + k] = sigma[k, j]
            A[row, N * N + i] = -1.0
            b[row] = 1.0 if i == j else 0.0
            row += 1
    for i in range(N):
        for k in range(N):
            A[row, i * N + k] = 1.0
        row += 1
    if np.linalg.cond(A) > 1e12:
        raise SingularSystem("alpha/gamma system is singular")
    x = np.linalg.solve(A, b)
    return x[:N * N].reshape(N, N), x[N * N:].copy()


def gamma_rhs(alpha, gamma, sigma, i, k, l, m):
    """Gamma_{i,k,l,m} of Eq. 14."""
    return -6.0 * (alpha[i, k] * (sigma[k, l] + sigma[k, m])
                   + alpha[i, l] * (sigma[k, l] + sigma[l, m])
                   + alpha[i, m] * (sigma[k, m] + sigma[l, m])
                   - gamma[i])


def _solve_small(A, b):
    if A.shape[0] == 0:
        return np.zeros(0)
    if np.linalg.cond(A) > 1e12:
        raise SingularSystem("alpha sub-matrix is singular")
    return np.linalg.solve(A, b)


def lambda_table(alpha, gamma, sigma):
    """Lambda_{j; j,k,l,m} for every triple k < l < m (Eqs. 14-15).

    For a triple, the rows and columns are the N - 3 components outside it;
    the matrix is that sub-matrix of alpha and the right-hand side is Gamma.
    Returns {(k, l, m): {j: Lambda}}.
    """
    N = alpha.shape[0]
    out = {}
    for k, l, m in itertools.combinations(range(N), 3):
        R = [j for j in range(N) if j not in (k, l, m)]
        A = alpha[np.ix_(R, R)]
        b = np.array([gamma_rhs(alpha, gamma, sigma, i, k, l, m) for i in R])
        sol = _solve_small(A, b)
        out[(k, l, m)] = {j: sol[a] for a, j in enumerate(R)}
    return out


def theta_table(alpha):
    """Theta_{kl; j; m} for every pair k < l and every m outside it (Eqs. 18-19).

    Rows and columns are the components outside {k, l, m}; the right-hand side
    is 2 alpha_{i m}.  Returns {(k, l, m): {j: Theta}}.
    """
    N = alpha.shape[0]
    out = {}
    for k, l in itertools.combinations(range(N), 2):
        for m in range(N):
            if m in (k, l):
                continue
            R = [j for j in range(N) if j not in (k, l, m)]
            A = alpha[np.ix_(R, R)]
            b = np.array([2.0 * alpha[i, m] for i in R])
            sol = _solve_small(A, b)
            out[(k, l, m)] = {j: sol[a] for a, j in enumerate(R)}
    return out


def spreading_parameters(sigma):
    """S_{ij;k} = sigma_ij - sigma_ik - sigma_jk for distinct i, j, k (Eq. 16)."""
    N = sigma.shape[0]
    out = {}
    for i, j, k in itertools.permutations(range(N), 3):
        out[(i, j, k)] = sigma[i, j] - sigma[i, k] - sigma[j, k]
    return out


def default_omega(sigma):
    """Omega = 0 when every spreading parameter is negative, else 1/90 (Sec. II, Eq. 17)."""
    S = spreading_parameters(np.asarray(sigma, dtype=np.float64))
    if not S or max(S.values()) < 0.0:
        return 0.0
    return 1.0 / 90.0


class Tables:
    """Everything Sec. II derives from (sigma, D, Omega) once per simulation."""

    def __init__(self, sigma, D=4.0, omega=float("nan")):
        self.sigma = np.asarray(sigma, dtype=np.float64)
        self.N = self.sigma.shape[0]
        self.D = float(D)
        self.omega = default_omega(self.sigma) if math.isnan(omega) else float(omega)
        self.beta, self.kappa = beta_kappa(self.sigma, self.D)
        self.alpha, self.gamma = alpha_gamma(self.sigma)
        self.lam = lambda_table(self.alpha, self.gamma, self.sigma)
        self.theta = theta_table(self.alpha) if self.omega != 0.0 else {}
        self._factored = None

    # -- chemical potential and the two correction terms ---------------------

    def mu_bulk(self, C):
        """dE_B/dC_j = sum_{k != j} beta_jk (f'(C_j) - f'(C_j + C_k)) (Eq. 7, bulk part)."""
        N = self.N
        out = np.zeros(C.shape)
        for j in range(N):
            for k in range(N):
                if k != j:
                    out[j] += self.beta[j, k] * (f_well_prime(C[j]) - f_well_prime(C[j] + C[k]))
        return out

    def mu(self, C, lapC):
        """mu_j of Eq. 7: the bulk part plus sum_{k != j} kappa_jk lap C_k."""
        out = self.mu_bulk(C)
        for j in range(self.N):
            for k in range(self.N):
                if k != j:
                    out[j] += self.kappa[j, k] * lapC[k]
        return out

    def phi(self, C):
        """phi_j = 12/D sum_{k<l<m, none = j} Lambda_{j;jklm} C_k C_l C_m (Eq. 13)."""
        out = np.zeros(C.shape)
        for (k, l, m), lam in self.lam.items():
            prod = C[k] * C[l] * C[m]
            for j, val in lam.items():
                out[j] += (12.0 / self.D) * val * prod
        return out

    def xi(self, C):
        """xi_j of Eq. 17 (zero when Omega = 0)."""
        out = np.zeros(C.shape)
        if self.omega == 0.0:
            return out
        N = self.N
        for j in range(N):
            for k, l in itertools.combinations(range(N), 2):
                if j in (k, l):
                    continue
                inner = 2.0 * C[j]
                for m in range(N):
                    if m in (j, k, l):
                        continue
                    inner = inner - self.theta[(k, l, m)][j] * C[m]
                out[j] += (12.0 / self.D) * self.omega * C[k] ** 2 * C[l] ** 2 * inner
        return out

    def flux_potential(self, C, lapC, with_phi=True):
        """S_i = sum_j alpha_ij (mu_j + phi_j + xi_j), Eq. 12, evaluated as written."""
        pot = self.mu(C, lapC) + self.xi(C)
        if with_phi:
            pot = pot + self.phi(C)
        return np.tensordot(self.alpha, pot, axes=(1, 0))

    def bulk_flux_potential(self, C, with_phi=True):
        """Bulk part of Eq. 12 (no Laplacian terms)."""
        pot = self.mu_bulk(C) + self.xi(C)
        if with_phi:
            pot = pot + self.phi(C)
        return np.tensordot(self.alpha, pot, axes=(1, 0))

    # -- factored form -------------------------------------------------------

    def polynomials(self):
        """Monomial expansion of the bulk flux potential, one Poly per component.

        Returns (cubic, quintic): cubic[i] = sum_j alpha_ij (dE_B/dC_j + phi_j)
        and quintic[i] = sum_j alpha_ij xi_j, in the variables C_0..C_{N-1}.
        """
        N = self.N
        Cv = [Poly.var(N, i) for i in range(N)]

        def fp(L):
            return 2.0 * L - 6.0 * (L ** 2) + 4.0 * (L ** 3)

        mu_b = []
        for j in range(N):
            p = Poly(N)
            for k in range(N):
                if k != j:
                    p = p + self.beta[j, k] * (fp(Cv[j]) - fp(Cv[j] + Cv[k]))
            mu_b.append(p)
        phi = [Poly(N) for _ in range(N)]
        for (k, l, m), lam in self.lam.items():
            prod = Cv[k] * Cv[l] * Cv[m]
            for j, val in lam.items():
                phi[j] = phi[j] + (12.0 / self.D) * val * prod
        xi = [Poly(N) for _ in range(N)]
        if self.omega != 0.0:
            for j in range(N):
                for k, l in itertools.combinations(range(N), 2):
                    if j in (k, l):
                        continue
                    inner = 2.0 * Cv[j]
                    for m in range(N):
                        if m not in (j, k, l):
                            inner = inner - self.theta[(k, l, m)][j] * Cv[m]
                    xi[j] = xi[j] + (12.0 / self.D) * self.omega * (Cv[k] ** 2) * (Cv[l] ** 2) * inner
        cubic, quintic = [], []
        for i in range(N):
            c = Poly(N)
            q = Poly(N)
            for j in range(N):
                c = c + self.alpha[i, j] * (mu_b[j] + phi[j])
                q = q + self.alpha[i, j] * xi[j]
            cubic.append(c)
            quintic.append(q)
        return cubic, quintic

    def factored(self, rtol=1e-10):
        """q_i with bulk S_i = C_i q_i(C) on the simplex (the factored form).

        The cubic part is made homogeneous of degree 3 with powers of
        sum_k C_k (exact on the simplex); every monomial free of C_i must then
        vanish, since a homogeneous polynomial that is zero on the face
        C_i = 0 of the simplex is zero.  The xi part is already a multiple of
        C_i.  Leftover coefficients above rtol times the largest one mean the
        Lambda or Theta solve did not cancel the flux, and raise.
        Returns (q2, q4, residual): lists of Poly of degree 2 and 4.
        """
        if self._factored is not None:
            return self._factored
        cubic, quintic = self.polynomials()
        q2, q4, resid = [], [], 0.0
        for i in range(self.N):
            h = cubic[i].homogenise(3)
            qi, rest = h.split_by_var(i)
            scale = max(h.max_abs_coeff(), 1e-300)
            r = rest.max_abs_coeff() / scale
            q5, rest5 = quintic[i].split_by_var(i)
            if quintic[i].terms:
                r = max(r, rest5.max_abs_coeff() / max(quintic[i].max_abs_coeff(), 1e-300))
            resid = max(resid, r)
            if r > rtol:
                raise SingularSystem(f"flux potential of component {i} is not divisible by C_{i} (residual {r:.3e})")
            q2.append(qi)
            q4.append(q5)
        self._factored = (q2, q4, resid)
        return self._factored

    def flux_potential_factored(self, C, lapC):
        """S_i = C_i (q2_i(C) + q4_i(C)) + (3 D / 4) lap C_i, equal to Eq. 12 on the simplex.

        The gradient part of Eq. 12 is sum_j alpha_ij sum_k kappa_jk lap C_k =
        (3D/4) (lap C_i + gamma_i lap sum_k C_k) by Eq. 8, and lap sum_k C_k = 0
        on the simplex.  An absent component (C_i = 0 on the stencil) gets
        S_i = 0.0 exactly.
        """
        q2, q4, _ = self.factored()
        out = np.zeros(C.shape)
        for i in range(self.N):
            q = q2[i](C)
            if q4[i].terms:
                q = q + q4[i](C)
            out[i] = C[i] * q + 0.75 * self.D * lapC[i]
        return out
