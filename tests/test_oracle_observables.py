"""Pins of the oracle's field observables on synthetic fields whose answer is fixed by construction:
the lens angle of Sec. IV A (circles fitted to the C = 0.5 contour, tangents at the triple points)
and the Laplace pressure jump of a droplet."""
import math

import numpy as np
import pytest

from oracle import observables


def _smooth_step(d):
    # 1/2 (1 + tanh(d / 2)): the interface profile of width 2 lu used for every initial field
    return 0.5 * (1.0 + np.tanh(0.5 * d))


def _lens(nx, ny, theta_up, theta_lo, a, xc, yc):
    """A lens whose interior angle at both triple points is theta_up + theta_lo (degrees).

    The triple points sit at (xc -/+ a, yc).  The upper arc meets the chord y = yc at theta_up:
    a circle through both triple points with its centre a cot(theta_up) below the chord, radius
    a / sin(theta_up); the lower arc likewise at theta_lo from above.  The lens is the
    intersection of the two discs, each edge smoothed by the tanh profile."""
    tu, tl = math.radians(theta_up), math.radians(theta_lo)
    c_up = yc - a / math.tan(tu)
    c_lo = yc + a / math.tan(tl)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    d_up = a / math.sin(tu) - np.hypot(x - xc, y - c_up)
    d_lo = a / math.sin(tl) - np.hypot(x - xc, y - c_lo)
    return _smooth_step(d_up) * _smooth_step(d_lo)


@pytest.mark.parametrize("theta", [53.5, 102.6, 147.7])      # Table 1 rows 1, 4 and 9 (Eq. 51)
@pytest.mark.parametrize("split", [0.5, 0.35])               # symmetric and asymmetric lenses
@pytest.mark.parametrize("grid", [(300, 150, 40.0), (128, 96, 20.0), (64, 64, 14.0)])
def test_lens_angle_recovers_the_constructed_angle(theta, split, grid):
    nx, ny, a = grid
    C = _lens(nx, ny, theta * split, theta * (1.0 - split), a, nx / 2 - 0.2, ny / 2 - 0.33)
    assert abs(observables.lens_angle(C) - theta) < 0.5


def test_lens_angle_of_a_mirrored_lens_is_unchanged():
    C = _lens(160, 100, 30.0, 75.0, 30.0, 79.6, 50.2)
    a0 = observables.lens_angle(C)
    assert abs(a0 - 105.0) < 0.5
    assert abs(observables.lens_angle(C[::-1]) - a0) < 1e-9       # upside down: arcs swap roles
    assert abs(observables.lens_angle(C[:, ::-1]) - a0) < 0.05    # left-right mirror


@pytest.mark.parametrize("R", [12.0, 20.0, 31.0])
def test_laplace_pressure_of_a_step_in_pressure(R):
    # P = P_in inside a disc of radius R and P_out outside, the drop field a tanh disc: the jump
    # is recovered exactly (the margin keeps both averages off the interface), and R from the
    # drop's area: a disc smoothed by 1/2 (1 + tanh(d / 2)) has area pi R^2 + pi^3 / 3 (the
    # profile's first moment about its midpoint is -pi^2 / 6), so R_eff = sqrt(R^2 + pi^2 / 3)
    n = 128
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    xc, yc = 63.3, 64.1
    r = np.hypot(x - xc, y - yc)
    drop = _smooth_step(R - r)
    P = np.where(r < R, 0.3042, 0.3)
    dP, Reff = observables.laplace_pressure(P, drop)
    assert abs(dP - 0.0042) < 1e-12
    assert abs(Reff - math.sqrt(R * R + math.pi ** 2 / 3.0)) < 1e-4
