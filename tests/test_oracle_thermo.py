"""Pins of the oracle's Sec. II code against what the paper and the mathematics fix."""
import itertools
import math

import numpy as np
import pytest

import nfe_workloads as W
from oracle import thermo


def _rng(seed=7):
    return np.random.default_rng(seed)


def test_beta_kappa_reproduce_width_and_tension():
    # Sec. II: D = sqrt(8 kappa / beta) and sigma = sqrt(2 kappa beta / 9).
    sigma = np.array([[0.0, 0.007], [0.007, 0.0]])
    for D in (3.0, 4.0, 6.0):
        beta, kappa = thermo.beta_kappa(sigma, D)
        assert math.isclose(math.sqrt(8 * kappa[0, 1] / beta[0, 1]), D, rel_tol=1e-14)
        assert math.isclose(math.sqrt(2 * kappa[0, 1] * beta[0, 1] / 9), 0.007, rel_tol=1e-14)


def test_planar_interface_excess_energy_equals_sigma():
    # The excess free energy per unit area of the D = 4 tanh profile must be sigma_12
    # (Sec. II, below Eq. 5).  Quadrature of E_B + E_I (Eq. 5) across a binary interface.
    sig = 0.0063
    D = 4.0
    beta, kappa = thermo.beta_kappa(np.array([[0, sig], [sig, 0]]), D)
    x = np.linspace(-60, 60, 240001)
    c = 0.5 * (1 + np.tanh(2 * x / D))
    dc = (1.0 / D) / np.cosh(2 * x / D) ** 2
    C = np.stack([c, 1 - c])
    EB = thermo.bulk_energy(C, beta)
    grad = np.zeros((2, 3, x.size))
    grad[0, 0] = dc
    grad[1, 0] = -dc
    EI = thermo.interface_energy(grad, kappa)
    total = np.trapezoid(EB + EI, x)
    assert abs(total - sig) / sig < 1e-8


def test_alpha_binary_closed_form():
    # Eqs. 8-9 for N = 2 solved by hand: alpha = (1 / (2 s)) [[-1, 1], [1, -1]], gamma = -1/2.
    s = 0.0081
    a, g = thermo.alpha_gamma(np.array([[0, s], [s, 0]]))
    np.testing.assert_allclose(a, np.array([[-1, 1], [1, -1]]) / (2 * s), rtol=1e-13)
    np.testing.assert_allclose(g, [-0.5, -0.5], rtol=1e-13)


@pytest.mark.parametrize("N", [3, 4, 5, 6, 7, 8])
def test_alpha_against_projected_inverse(N):
    # Eliminating gamma from Eqs. 8-9 by hand: alpha = S^-1 - (S^-1 1)(1^T S^-1) / (1^T S^-1 1),
    # gamma = -(S^-1 1) / (1^T S^-1 1).  The oracle solves the full (N^2+N) system instead.
    rng = _rng(N)
    sig = W.random_sigma(rng, N)
    a, g = thermo.alpha_gamma(sig)
    Si = np.linalg.inv(sig)
    one = np.ones(N)
    u = Si @ one
    a_ref = Si - np.outer(u, u) / (one @ u)
    np.testing.assert_allclose(a, a_ref, rtol=1e-10, atol=1e-10 * np.abs(a_ref).max())
    np.testing.assert_allclose(g, -u / (one @ u), rtol=1e-10)
    np.testing.assert_allclose(a, a.T, atol=1e-10 * np.abs(a).max())
    np.testing.assert_allclose(a.sum(axis=0), 0, atol=1e-10 * np.abs(a).max())
    np.testing.assert_allclose(a @ sig, np.eye(N) + np.outer(g, one), atol=1e-11)


def _eq10_bracket(T, C, i):
    """Bracket of Eq. 10 (the bulk flux potential without phi), for component i."""
    D = T.D
    out = -C[i] * (1 - 3 * C[i] + 2 * C[i] ** 2)
    a, s, g = T.alpha, T.sigma, T.gamma
    for j, k, l in itertools.combinations(range(T.N), 3):
        coef = (a[i, j] * (s[j, k] + s[j, l]) + a[i, k] * (s[j, k] + s[k, l])
                + a[i, l] * (s[j, l] + s[k, l]) - g[i])
        out = out + 6 * coef * C[j] * C[k] * C[l]
    return 12.0 / D * out


@pytest.mark.parametrize("N", [3, 4, 5, 6])
def test_bulk_flux_matches_eq10(N):
    # Eq. 10 prints the bulk flux potential sum_j alpha_ij mu_{j,b} on the simplex in closed
    # form.  The oracle builds it from Eq. 7 and the alpha of Eqs. 8-9; the two must agree.
    rng = _rng(100 + N)
    T = thermo.Tables(W.random_sigma(rng, N), omega=0.0)
    C = W.random_simplex_points(rng, N, 200).T
    direct = T.bulk_flux_potential(C, with_phi=False)
    for i in range(N):
        np.testing.assert_allclose(direct[i], _eq10_bracket(T, C, i), rtol=1e-9, atol=1e-12)


def test_three_components_need_no_phi():
    # Sec. II, Eq. 11: for N = 3 the flux of an absent component vanishes without phi.
    rng = _rng(3)
    T = thermo.Tables(W.random_sigma(rng, 3), omega=0.0)
    assert all(len(v) == 0 for v in T.lam.values())
    for absent in range(3):
        C = W.random_simplex_points(rng, 3, 100, absent=absent).T
        assert np.abs(T.bulk_flux_potential(C, with_phi=False)[absent]).max() < 1e-14


@pytest.mark.parametrize("N", [4, 5, 6, 7, 8])
def test_phi_gives_reduction_consistency(N):
    # Sec. II, Eqs. 12-15: with phi the bulk potential of an absent component is zero on the
    # simplex (no nucleation); without phi it is O(1) at points where >= 3 others are present.
    rng = _rng(200 + N)
    T = thermo.Tables(W.random_sigma(rng, N), omega=0.0)
    for absent in (0, N // 2, N - 1):
        C = W.random_simplex_points(rng, N, 100, absent=absent).T
        with_phi = T.bulk_flux_potential(C)[absent]
        without = T.bulk_flux_potential(C, with_phi=False)[absent]
        assert np.abs(with_phi).max() < 1e-13
        assert np.abs(without).max() > 1e-3


@pytest.mark.parametrize("N", [3, 4, 5, 6])
def test_xi_part_is_a_multiple_of_Ci(N):
    # Eqs. 17-19: Theta is chosen so that sum_j alpha_ij xi_j vanishes where C_i = 0,
    # for any C (not only on the simplex).
    rng = _rng(300 + N)
    T = thermo.Tables(W.random_sigma(rng, N), omega=1.0 / 90.0)
    for i in range(N):
        C = rng.uniform(0, 1, size=(N, 50))
        C[i] = 0.0
        X = np.tensordot(T.alpha, T.xi(C), axes=(1, 0))[i]
        scale = np.abs(np.tensordot(T.alpha, T.xi(rng.uniform(0, 1, size=(N, 50))), axes=(1, 0))).max()
        assert np.abs(X).max() < 1e-12 * max(scale, 1e-30)


def test_spreading_and_default_omega():
    # Eq. 16 and the rule below Eq. 17: Omega = 0 when all spreading parameters are negative.
    s = np.full((3, 3), 0.005)
    np.fill_diagonal(s, 0)
    assert thermo.default_omega(s) == 0.0
    s[0, 1] = s[1, 0] = 0.012
    sp = thermo.spreading_parameters(s)
    assert math.isclose(sp[(0, 1, 2)], 0.012 - 0.005 - 0.005)
    assert thermo.default_omega(s) == 1.0 / 90.0


@pytest.mark.parametrize("N,omega", [(2, 0.0), (3, 0.0), (4, 0.0), (4, 1 / 90), (5, 1 / 90), (7, 0.0), (8, 1 / 90)])
def test_factored_equals_literal_on_simplex(N, omega):
    # The factored S_i = C_i q_i + (3D/4) lap C_i equals Eq. 12 on the simplex, and is exactly
    # 0.0 for an absent component whose Laplacian is zero.
    rng = _rng(400 + N)
    T = thermo.Tables(W.random_sigma(rng, N), omega=omega)
    C = W.random_simplex_points(rng, N, 300).T
    lap = rng.normal(scale=0.05, size=C.shape)
    lap -= lap.mean(axis=0)
    lit = T.flux_potential(C, lap)
    fac = T.flux_potential_factored(C, lap)
    np.testing.assert_allclose(fac, lit, rtol=0, atol=1e-12 * np.abs(lit).max())
    _, _, resid = T.factored()
    assert resid < 1e-12
    C0 = W.random_simplex_points(rng, N, 50, absent=N - 1).T
    lap0 = np.zeros_like(C0)
    assert (T.flux_potential_factored(C0, lap0)[N - 1] == 0.0).all()


def test_factored_rejects_broken_lambda():
    # A wrong Lambda leaves monomials free of C_i behind: the factorisation must refuse it.
    rng = _rng(11)
    T = thermo.Tables(W.random_sigma(rng, 5), omega=0.0)
    key = next(iter(T.lam))
    j = next(iter(T.lam[key]))
    T.lam[key][j] *= 1.01
    with pytest.raises(thermo.SingularSystem):
        T.factored()
