"""The oracle's domain size L_i (Sec. IV, the equation for L_i) against what fixes it:
a direct DFT on a tiny grid, patterns with a single wavenumber (closed form L = 2 pi / |k|),
and exact invariances."""
import math

import numpy as np

from oracle import observables


def _two(lam):
    lam = np.asarray(lam, dtype=np.float64)
    C = np.zeros((2,) + lam.shape)
    C[0] = lam
    C[1] = 1.0 - lam
    return C


def _direct_L(lam):
    # L = 2 pi sum_{k != 0} |F(k)|^2 / sum_{k != 0} |k| |F(k)|^2 with F summed site by site
    nz, ny, nx = lam.shape
    num = den = 0.0
    zs, ys, xs = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for mz in range(nz):
        for my in range(ny):
            for mx in range(nx):
                if mx == my == mz == 0:
                    continue
                ph = 2 * math.pi * (mx * xs / nx + my * ys / ny + mz * zs / nz)
                F = np.sum(lam * np.exp(-1j * ph))
                fold = lambda m, n: (m - n if m > n / 2 else m) / n
                kk = 2 * math.pi * math.sqrt(fold(mx, nx) ** 2 + fold(my, ny) ** 2 + fold(mz, nz) ** 2)
                num += abs(F) ** 2
                den += kk * abs(F) ** 2
    return 2 * math.pi * num / den


def test_domain_size_matches_a_direct_dft():
    rng = np.random.default_rng(3)
    for shape in ((1, 6, 10), (3, 4, 5)):
        C = rng.uniform(0.0, 1.0, size=(2,) + shape)
        L, _ = observables.domain_size(C)
        lam = (C[0] >= 0.5).astype(np.float64)
        assert abs(L[0] - _direct_L(lam)) <= 1e-12 * L[0]


def test_single_wavenumber_patterns_give_two_pi_over_k():
    # period-4 stripes (1, 1, 0, 0): only |k| = 2 pi / 4; a checkerboard: only |k| = pi sqrt(2)
    x = np.arange(64)
    stripes = np.broadcast_to((x % 4 < 2).astype(float), (1, 8, 64))
    L, mean = observables.domain_size(_two(stripes))
    assert np.allclose(L, 4.0, rtol=1e-13) and abs(mean - 4.0) < 1e-12
    y, xx = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
    board = ((xx + y) % 2 == 0).astype(float)[None]
    L, _ = observables.domain_size(_two(board))
    assert np.allclose(L, math.sqrt(2.0), rtol=1e-13)


def test_domain_size_invariances():
    # a periodic shift and a quarter turn leave every |F(k)| and |k| as they were; the two
    # complementary components have the same spectrum at k != 0
    rng = np.random.default_rng(5)
    lam = (rng.uniform(size=(1, 24, 24)) > 0.5).astype(float)
    L0, _ = observables.domain_size(_two(lam))
    L1, _ = observables.domain_size(_two(np.roll(lam, (5, -7), axis=(1, 2))))
    L2, _ = observables.domain_size(_two(np.rot90(lam, axes=(1, 2))))
    assert np.allclose(L1, L0, rtol=1e-12) and np.allclose(L2, L0, rtol=1e-12)
    assert abs(L0[0] - L0[1]) < 1e-12 * L0[0]


def test_uniform_phase_has_no_domain_size():
    C = np.zeros((2, 1, 8, 8))
    C[0] = 1.0
    L, mean = observables.domain_size(C)
    assert np.isnan(L).all() and np.isnan(mean)
