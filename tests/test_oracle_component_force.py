"""The oracle's body force on one component, F += C_c F_c (the PaLS study of Sec. V pushes only
the droplet of fluid 2), against what fixes it: the momentum it adds per step over a periodic
domain is F_c times the mass of component c, and in a pure phase of c it is the uniform body
force of Eq. 2."""
import numpy as np

import nfe_workloads as W
from oracle import lbm


def _momentum(prm, st):
    return np.einsum("ka,kn->a", prm.lat.e.astype(float), st.f.reshape(prm.lat.Q, -1))


def test_momentum_gain_is_the_force_times_the_component_mass():
    p = W.janus_2d(nx=48, ny=40, radius=9, offset=11)
    p["component_force"] = (3e-7, -2e-7, 0.0)
    p["component_force_index"] = 1
    prm = lbm.Params(p)
    st = lbm.init_state(prm, p["C0"])
    for _ in range(8):
        C = lbm.components(prm, st.g)
        mass = C[1].sum()
        j0 = _momentum(prm, st)
        st = lbm.step(prm, st)
        gain = _momentum(prm, st) - j0
        # F_s sums to zero over a periodic domain (Eq. 34), so only the component force remains
        np.testing.assert_allclose(gain, np.array([3e-7, -2e-7, 0.0]) * mass, rtol=1e-9, atol=1e-18)


def test_pure_phase_of_the_component_feels_the_uniform_body_force():
    a = W.planar_2d(nx=6, ny=24)
    C = np.zeros_like(a["C0"])
    C[1] = 1.0
    a["C0"] = C
    b = dict(a)
    a["body_force"] = (4e-6, 1e-6, 0.0)
    b["component_force"] = (4e-6, 1e-6, 0.0)
    b["component_force_index"] = 1
    pa, pb = lbm.Params(a), lbm.Params(b)
    sa = lbm.run(pa, lbm.init_state(pa, C), 12)
    sb = lbm.run(pb, lbm.init_state(pb, C), 12)
    np.testing.assert_allclose(sb.f, sa.f, rtol=0, atol=1e-18)
    assert np.abs(_momentum(pa, sa)).max() > 1e-6
