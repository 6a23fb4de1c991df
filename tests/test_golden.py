"""The oracle's observables against numbers the paper prints (tests/golden/)."""
import os

import numpy as np

from oracle import observables

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_table1_neumann_theory_angles():
    # Sec. IV A, Table 1: the theory columns follow from Eq. 51 with the lens fluid as phase k
    # (interior angle) and fluid 1 as phase k (exterior angle), printed to 0.1 degree.
    rows = np.loadtxt(os.path.join(GOLD, "table1_neumann.txt"))
    assert rows.shape == (9, 10)
    for s12, s13, s14, s23, s24, s34, th_in, th_out, _, _ in rows:
        assert abs(observables.neumann_angle(s12, s13, s23) - th_in) <= 0.051
        assert abs(observables.neumann_angle(s23, s12, s13) - th_out) <= 0.051
        # the angles at a triple point add up to 360 degrees
        total = (observables.neumann_angle(s12, s13, s23) + observables.neumann_angle(s23, s12, s13)
                 + observables.neumann_angle(s13, s12, s23))
        assert abs(total - 360.0) < 1e-9


def _read_poiseuille():
    vals = {}
    with open(os.path.join(GOLD, "poiseuille_constants.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                key, *rest = line.split()
                vals[key] = [float(x) for x in rest]
    return vals


def test_poiseuille_constants_printed_sign():
    # Sec. IV C: with the printed sign of Eq. 53 (eta v'' = +F) the system of Eq. 58 gives the
    # printed A and B_i (three significant figures).
    g = _read_poiseuille()
    eta = (np.array(g["tau"]) - 0.5) / 3.0
    sol = observables.poiseuille_constants(g["interfaces"], eta, g["F"][0], g["W"][0], sign=+1.0)
    np.testing.assert_allclose(sol[0], g["A"][0], rtol=5e-3)
    np.testing.assert_allclose(sol[1:], g["B"], rtol=5e-3, atol=1e-7)


def test_poiseuille_profile_solves_its_ode():
    # The profile is continuous, zero at both walls, has continuous shear stress eta v' and
    # satisfies eta_i v'' = sign F in every layer.
    g = _read_poiseuille()
    eta = (np.array(g["tau"]) - 0.5) / 3.0
    W, F = g["W"][0], g["F"][0]
    for sign in (+1.0, -1.0):
        prof = lambda x: observables.poiseuille_profile(x, g["interfaces"], eta, F, W, sign)
        assert abs(prof([0.0])[0]) < 1e-15 and abs(prof([W - 1e-12])[0]) < 1e-12
        for i, xi in enumerate(g["interfaces"]):
            h = 1e-6
            l, r = prof([xi - h])[0], prof([xi + h])[0]
            assert abs(l - r) < 1e-9
            dl = (prof([xi - h])[0] - prof([xi - 2 * h])[0]) / h
            dr = (prof([xi + 2 * h])[0] - prof([xi + h])[0]) / h
            assert abs(eta[i] * dl - eta[i + 1] * dr) < 1e-9
        x = np.array([30.0, 90.0, 150.0, 210.0, 270.0, 330.0])
        h = 1e-2
        d2 = (prof(x + h) - 2 * prof(x) + prof(x - h)) / h ** 2
        np.testing.assert_allclose(eta * d2, sign * F, rtol=1e-4)
