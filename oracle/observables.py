"""Sec. IV observables: Neumann angles, layered Poiseuille flow, Laplace pressure, domain size.

Oracle code (test infrastructure only).  Plain numpy in float64.
"""
from __future__ import annotations

import math

import numpy as np


def neumann_angle(sigma_ij, sigma_ik, sigma_jk):
    """Angle (degrees) inside phase k at an i-j-k triple point (Eq. 51).

    Eq. 51 gives cos(pi - theta) = -(sigma_ij^2 - sigma_ik^2 - sigma_jk^2) /
    (2 sigma_ik sigma_jk) for the angle between the i-k and j-k interfaces.
    """
    c = (sigma_ij ** 2 - sigma_ik ** 2 - sigma_jk ** 2) / (2.0 * sigma_ik * sigma_jk)
    return math.degrees(math.pi - math.acos(-c))


def poiseuille_constants(interfaces, eta, F, W, sign=+1.0):
    """Integration constants (A, B_1..B_L) of the layered profile (Eqs. 53-58).

    Layer i obeys eta_i v'' = sign * F (the paper prints sign = +1, Eq. 53);
    Eq. 56 then gives v_i(x) = sign F x^2 / (2 eta_i) + A x / eta_i + B_i.
    Conditions: v_1(0) = 0, v_L(W) = 0 and continuity of v at each interface
    x_i (continuity of shear stress is built into the common A).  Returns
    the solution of the (L+1) x (L+1) system of Eq. 58.
    """
    eta = np.asarray(eta, dtype=np.float64)
    L = len(eta)
    x = np.asarray(interfaces, dtype=np.float64)
    M = np.zeros((L + 1, L + 1))
    b = np.zeros(L + 1)
    # unknowns: [A, B_1, ..., B_L]
    M[0, 1] = 1.0                                   # v_1(0) = 0
    M[1, 0] = W / eta[L - 1]
    M[1, L] = 1.0
    b[1] = -sign * F * W * W / (2.0 * eta[L - 1])   # v_L(W) = 0
    for i in range(L - 1):
        xi = x[i]
        # v_i(x_i) - v_{i+1}(x_i) = 0
        M[2 + i, 0] = xi / eta[i] - xi / eta[i + 1]
        M[2 + i, 1 + i] = 1.0
        M[2 + i, 2 + i] = -1.0
        b[2 + i] = -sign * F * xi * xi * (1.0 / (2.0 * eta[i]) - 1.0 / (2.0 * eta[i + 1]))
    return np.linalg.solve(M, b)


def poiseuille_profile(xs, interfaces, eta, F, W, sign=+1.0):
    """v(x) of Eq. 56 at the points xs (0 <= x <= W)."""
    sol = poiseuille_constants(interfaces, eta, F, W, sign)
    A, B = sol[0], sol[1:]
    eta = np.asarray(eta, dtype=np.float64)
    xs = np.asarray(xs, dtype=np.float64)
    layer = np.searchsorted(np.asarray(interfaces, dtype=np.float64), xs, side="right")
    return sign * F * xs ** 2 / (2.0 * eta[layer]) + A * xs / eta[layer] + B[layer]


def laplace_pressure(P, C_drop, margin=4.0):
    """Pressure jump across a 2-D droplet and its radius from the drop's area.

    R = sqrt(sum C_drop / pi); P_in is the mean of P over r < R - margin and
    P_out the mean over r > R + margin, r measured from the drop's centroid.
    Returns (P_in - P_out, R).
    """
    P = np.asarray(P, dtype=np.float64).reshape(C_drop.shape[-2:])
    Cd = np.asarray(C_drop, dtype=np.float64).reshape(P.shape)
    ny, nx = P.shape
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    mass = Cd.sum()
    xc, yc = (Cd * x).sum() / mass, (Cd * y).sum() / mass
    R = math.sqrt(mass / math.pi)
    r = np.hypot(x - xc, y - yc)
    inside = r < R - margin
    outside = r > R + margin
    return P[inside].mean() - P[outside].mean(), R


def _fit_circle(px, py):
    """Algebraic least-squares circle through points: returns (xc, yc, R)."""
    A = np.column_stack([px, py, np.ones_like(px)])
    b = px * px + py * py
    sol, *_ = np.linalg.lstsq(A, b, rcond=None)
    xc, yc = sol[0] / 2.0, sol[1] / 2.0
    R = math.sqrt(sol[2] + xc * xc + yc * yc)
    return xc, yc, R


def lens_angle(C_lens, keep=0.6):
    """Interior angle (degrees) of a lens from the C = 0.5 contour of its phase.

    Sec. IV A: the top and bottom of the contour are fitted by two circles and
    the angle is taken from their tangents at the triple points.  Crossings are
    found column by column with linear interpolation; only the central `keep`
    fraction of the lens width enters the fits, away from the triple points.
    The lens is the intersection of the two discs, so its angle at a triple
    point is pi minus the angle between the two outward normals.
    """
    Cl = np.asarray(C_lens, dtype=np.float64)
    Cl = Cl.reshape(Cl.shape[-2:])
    ny, nx = Cl.shape
    cols, tops, bots = [], [], []
    for x in range(nx):
        col = Cl[:, x]
        if col.max() <= 0.5:
            continue
        above = np.nonzero(col > 0.5)[0]
        lo, hi = above[0], above[-1]
        if lo == 0 or hi == ny - 1:
            continue
        yb = lo - 1 + (0.5 - col[lo - 1]) / (col[lo] - col[lo - 1])
        yt = hi + (col[hi] - 0.5) / (col[hi] - col[hi + 1])
        cols.append(float(x))
        tops.append(yt)
        bots.append(yb)
    cols = np.array(cols)
    if len(cols) < 6:
        raise ValueError("lens too small to measure")
    mid, half = 0.5 * (cols.min() + cols.max()), 0.5 * (cols.max() - cols.min())
    sel = np.abs(cols - mid) <= keep * half
    c1 = _fit_circle(cols[sel], np.array(tops)[sel])     # upper arc
    c2 = _fit_circle(cols[sel], np.array(bots)[sel])     # lower arc
    d = math.hypot(c2[0] - c1[0], c2[1] - c1[1])
    # one intersection point of the two circles
    a = (c1[2] ** 2 - c2[2] ** 2 + d * d) / (2.0 * d)
    h = math.sqrt(max(c1[2] ** 2 - a * a, 0.0))
    ux, uy = (c2[0] - c1[0]) / d, (c2[1] - c1[1]) / d
    px, py = c1[0] + a * ux - h * uy, c1[1] + a * uy + h * ux
    n1 = np.array([px - c1[0], py - c1[1]]) / c1[2]
    n2 = np.array([px - c2[0], py - c2[1]]) / c2[2]
    psi = math.acos(max(-1.0, min(1.0, float(n1 @ n2))))
    return math.degrees(math.pi - psi)


def domain_size(C):
    """Domain size of every component (Sec. IV, the equation for L_i), with the mean over them.

    lambda_i = H(C_i - 1/2) (H(0) = 1); S_i(k) = |lambda_i(k)|^2 from the discrete Fourier
    transform over the grid taken as periodic; L_i = 2 pi sum_{k != 0} S_i(k) /
    sum_{k != 0} |k| S_i(k), the k-plane integrals of the circularly averaged S_i written
    as sums over the grid's modes, k = 2 pi m / n per axis.  C has shape (N, nz, ny, nx);
    returns (L array of N values, mean of the finite ones).
    """
    C = np.asarray(C, dtype=np.float64)
    shape = C.shape[1:]
    ks = np.meshgrid(*[2.0 * np.pi * np.fft.fftfreq(n) for n in shape], indexing="ij")
    kabs = np.sqrt(sum(k * k for k in ks))
    L = np.empty(C.shape[0])
    for i in range(C.shape[0]):
        lam = (C[i] >= 0.5).astype(np.float64)
        S = np.abs(np.fft.fftn(lam)) ** 2
        S.flat[0] = 0.0                                  # k = 0 is excluded
        den = np.sum(kabs * S)
        L[i] = 2.0 * np.pi * S.sum() / den if den > 0.0 else np.nan
    fin = L[np.isfinite(L)]
    return L, (fin.mean() if fin.size else np.nan)
