"""Pins of the oracle's Sec. III stepper: lattice identities, stencils, moments,
conservation, reduction consistency and the paper's benchmark physics."""
import math

import numpy as np
import pytest

import nfe_workloads as W
from oracle import lbm, observables, thermo


@pytest.mark.parametrize("q", [9, 19])
def test_lattice_isotropy(q):
    # Weights and velocities of Eqs. 20-21 (and the standard D3Q19 set): the moments
    # up to fourth order must be those of the Maxwellian with c_s^2 = 1/3.
    lat = lbm.Lattice(q)
    e, w = lat.e.astype(float), lat.w
    d = lat.dim
    assert math.isclose(w.sum(), 1.0, rel_tol=1e-15)
    np.testing.assert_allclose(w @ e, 0, atol=1e-16)
    M2 = np.einsum("k,ka,kb->ab", w, e, e)[:d, :d]
    np.testing.assert_allclose(M2, np.eye(d) / 3, atol=1e-15)
    M3 = np.einsum("k,ka,kb,kc->abc", w, e, e, e)
    np.testing.assert_allclose(M3, 0, atol=1e-15)
    M4 = np.einsum("k,ka,kb,kc,kd->abcd", w, e, e, e, e)[:d, :d, :d, :d]
    I = np.eye(d)
    ref = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I) + np.einsum("ad,bc->abcd", I, I)) / 9
    np.testing.assert_allclose(M4, ref, atol=1e-15)
    for k in range(q):
        assert (e[lat.opp[k]] == -e[k]).all()


def _prm(q, nx, ny, nz, walls=(False, False, False), N=2):
    sig = np.full((N, N), 0.005)
    np.fill_diagonal(sig, 0)
    return lbm.Params(W.base_params(q, nx, ny, nz, N, sig, 1.0, walls=walls))


@pytest.mark.parametrize("q", [9, 19])
def test_stencils_exact_on_polynomials(q):
    # Eqs. 35-36 are exact for linear fields (gradient) and quadratics (Laplacian) away
    # from the periodic seam.
    nz = 1 if q == 9 else 12
    prm = _prm(q, 12, 11, nz)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(11), np.arange(12), indexing="ij")
    lin = 0.3 * x - 0.7 * y + (0.2 * z if q == 19 else 0)
    quad = 0.5 * x * x + 0.25 * y * y + (0.125 * z * z if q == 19 else 0) + x * y
    g = lbm.grad(prm, lin.astype(float))
    lap = lbm.laplacian(prm, quad.astype(float))
    sl = (slice(1, -1) if q == 19 else slice(None), slice(1, -1), slice(1, -1))
    np.testing.assert_allclose(g[0][sl], 0.3, atol=1e-13)
    np.testing.assert_allclose(g[1][sl], -0.7, atol=1e-13)
    if q == 19:
        np.testing.assert_allclose(g[2][sl], 0.2, atol=1e-13)
    np.testing.assert_allclose(lap[sl], 1.0 + 0.5 + (0.25 if q == 19 else 0.0), atol=1e-12)


@pytest.mark.parametrize("q", [9, 19])
def test_periodic_gradient_sums_to_zero_and_wall_rule(q):
    rng = np.random.default_rng(1)
    nz = 1 if q == 9 else 6
    prm = _prm(q, 9, 7, nz)
    psi = rng.normal(size=prm.shape)
    g = lbm.grad(prm, psi)
    assert np.abs(g.reshape(3, -1).sum(axis=1)).max() < 1e-13
    assert abs(lbm.laplacian(prm, psi).sum()) < 1e-12
    # wall rule (Sec. III C): a constant field has no gradient or Laplacian next to a wall
    prmw = _prm(q, 9, 7, nz, walls=(False, True, q == 19))
    const = np.full(prmw.shape, 0.37)
    assert np.abs(lbm.grad(prmw, const)).max() == 0.0
    assert np.abs(lbm.laplacian(prmw, const)).max() == 0.0


@pytest.mark.parametrize("q", [9, 19])
def test_equilibria_moments(q):
    lat = lbm.Lattice(q)
    rng = np.random.default_rng(2)
    v = rng.normal(scale=0.05, size=(3, 20))
    if q == 9:
        v[2] = 0
    P = rng.normal(scale=1e-3, size=20)
    feq = lbm.f_equilibrium(lat, P, v)
    e = lat.e.astype(float)
    np.testing.assert_allclose(np.einsum("ka,kn->an", e, feq), v, atol=1e-16)
    # Eq. 38 applied to f^eq returns P (with F = 0)
    P_back = lbm.CS2 / (1 - lat.w[0]) * (feq[1:].sum(axis=0) + lbm.s_k(lat, v)[0])
    np.testing.assert_allclose(P_back, P, atol=1e-16)
    # Eq. 40: zeroth moment C (Eq. 41), first moment C v (advection of Eq. 3) and second
    # moment C v v - c_s^2 m S I, whose Chapman-Enskog limit is the flux of Eq. 12 with the
    # mobility of Eq. 43 and no extra diffusion of C.
    C = rng.uniform(0, 1, 20)
    S = rng.normal(size=20)
    m = 0.02
    geq = lbm.g_equilibrium(lat, C, v, S, m)
    np.testing.assert_allclose(geq.sum(axis=0), C, atol=1e-15)
    np.testing.assert_allclose(np.einsum("ka,kn->an", e, geq), C * v, atol=1e-15)
    d = lat.dim
    M2 = np.einsum("ka,kb,kn->abn", e, e, geq)[:d, :d]
    ref = np.einsum("an,bn->abn", C * v, v)[:d, :d] - (lbm.CS2 * m * S)[None, None, :] * np.eye(d)[:, :, None]
    np.testing.assert_allclose(M2, ref, atol=1e-15)
    # forcing of Eq. 30: zeroth moment 0, first moment F
    F = rng.normal(scale=1e-4, size=(3, 20))
    if q == 9:
        F[2] = 0
    Fk = lbm.forcing_terms(lat, v, F)
    np.testing.assert_allclose(Fk.sum(axis=0), 0, atol=1e-18)
    np.testing.assert_allclose(np.einsum("ka,kn->an", e, Fk), F, atol=1e-18)


@pytest.mark.parametrize("q", [9, 19])
def test_collision_adds_exactly_the_force_to_momentum(q):
    # TRT collision with the forcing split of Eq. 29 changes sum_k e_k f_k by exactly F.
    lat = lbm.Lattice(q)
    rng = np.random.default_rng(3)
    n = 30
    f = rng.normal(scale=1e-3, size=(q, n))
    F = rng.normal(scale=1e-5, size=(3, n))
    if q == 9:
        F[2] = 0
    e = lat.e.astype(float)
    v = np.einsum("ka,kn->an", e, f) + 0.5 * F
    P = rng.normal(scale=1e-3, size=n)
    op = 1 / rng.uniform(0.55, 1.5, n)
    om = 1 / rng.uniform(0.55, 1.5, n)
    post = lbm.collide_f(lat, f, P, v, F, op, om)
    dj = np.einsum("ka,kn->an", e, post) - np.einsum("ka,kn->an", e, f)
    np.testing.assert_allclose(dj, F, atol=1e-17)


def test_f0_never_matters():
    # f_0 feeds no moment (Eqs. 37-38) and pairs only with itself in TRT: either sign of the
    # k = 0 pressure term of Eq. 27 gives bitwise identical f_{k != 0} and g.
    p = W.lens_2d(nx=24, ny=20, radius=5)
    prm = lbm.Params(p)
    a = lbm.init_state(prm, p["C0"])
    b = lbm.init_state(prm, p["C0"])
    a = lbm.run(prm, a, 15, feq0_sign=-1.0)
    b = lbm.run(prm, b, 15, feq0_sign=+1.0)
    assert np.array_equal(a.f[1:], b.f[1:]) and np.array_equal(a.g, b.g)
    assert not np.array_equal(a.f[0], b.f[0])


@pytest.mark.parametrize("case", ["spinodal", "lens_walls", "janus3d"])
def test_mass_conserved(case):
    if case == "spinodal":
        p = W.spinodal_2d(nx=32, ny=24)
    elif case == "lens_walls":
        p = W.lens_2d(nx=32, ny=28, radius=6)
    else:
        p = W.janus_3d(n=16, radius=4)
    prm = lbm.Params(p)
    st = lbm.init_state(prm, p["C0"])
    m0 = lbm.diagnostics(prm, st)["mass"]
    st = lbm.run(prm, st, 40)
    m1 = lbm.diagnostics(prm, st)["mass"]
    np.testing.assert_allclose(m1, m0, rtol=0, atol=1e-13 * prm.shape[0] * prm.shape[1] * prm.shape[2])


@pytest.mark.parametrize("q", [9, 19])
def test_momentum_conserved_periodic(q):
    # Eq. 34 sums to zero over a periodic domain (grad E_B telescopes; the kappa term is a
    # commutator of circulant stencils), so the momentum changes only by the body force.
    if q == 9:
        p = W.janus_2d(nx=48, ny=40, radius=9, offset=11)
    else:
        p = W.janus_3d(n=16, radius=4)
    p["body_force"] = (2e-7, -1e-7, 0.0 if q == 9 else 3e-7)
    prm = lbm.Params(p)
    st = lbm.init_state(prm, p["C0"])
    n = np.prod(prm.shape)
    for _ in range(10):
        d0 = lbm.diagnostics(prm, st)
        assert np.abs(d0["force_sum"]).max() <= 1e-13 * d0["force_abs_sum"].sum()
        C = lbm.components(prm, st.g)
        mac = lbm.macroscopic(prm, C, st.f)
        j0 = np.einsum("ka,kn->a", prm.lat.e.astype(float), st.f.reshape(prm.lat.Q, -1))
        st = lbm.step(prm, st)
        j1 = np.einsum("ka,kn->a", prm.lat.e.astype(float), st.f.reshape(prm.lat.Q, -1))
        np.testing.assert_allclose(j1 - j0, mac["F"].reshape(3, -1).sum(axis=1), rtol=0,
                                   atol=1e-13 * (np.abs(mac["Fs"]).sum() + n * 1e-6))


def test_absent_component_stays_absent():
    # Sec. IV A: with phi the absent components stay at machine precision (literal Eq. 12) and
    # exactly 0.0 in the factored form; without phi the absent component nucleates at the
    # triple points of the other three.
    p = W.lens_2d(nx=40, ny=36, radius=8, N=3)
    N = 4
    C = np.zeros((N,) + p["C0"].shape[1:])
    C[:3] = p["C0"]
    sig = np.full((N, N), 0.005)
    np.fill_diagonal(sig, 0)
    sig[:3, :3] = p["sigma"]
    # the absent component must be an evolved one: the implicit C_0 = 1 - sum of the others
    # follows the compressible part of the LBM velocity field
    q = W.base_params(9, 40, 36, 1, N, sig, 1.0, walls=(False, True, False), m=0.05, omega_stab=0.0,
                      implicit=0)
    prm = lbm.Params(q)
    lit = lbm.run(prm, lbm.init_state(prm, C), 60)
    fac = lbm.run(prm, lbm.init_state(prm, C, flux_form="factored"), 60, flux_form="factored")
    nophi = lbm.run(prm, lbm.init_state(prm, C), 60, with_phi=False)
    assert np.abs(lbm.components(prm, lit.g)[3]).max() < 1e-14
    assert (lbm.components(prm, fac.g)[3] == 0.0).all()
    assert np.abs(lbm.components(prm, nophi.g)[3]).max() > 1e-6


def test_factored_and_literal_trajectories_agree():
    p = W.spinodal_2d(nx=24, ny=20, seed=5)
    prm = lbm.Params(p)
    a = lbm.run(prm, lbm.init_state(prm, p["C0"]), 100)
    b = lbm.run(prm, lbm.init_state(prm, p["C0"], flux_form="factored"), 100, flux_form="factored")
    # The two forms differ only by rounding in S_i; C agrees to ~1e-16.  f is a small,
    # decaying velocity/pressure signal (max ~5e-7 here, ~1e-5 at the start) computed from
    # C differences, so its error is bounded relative to its largest value over the run.
    Ca, Cb = lbm.components(prm, a.g), lbm.components(prm, b.g)
    assert np.abs(Ca - Cb).max() <= 1e-14
    assert np.abs(a.f - b.f).max() <= 1e-11 * np.abs(a.f).max()


@pytest.mark.slow
def test_planar_interface_keeps_tanh_profile():
    # Sec. II: the binary equilibrium profile is C = 1/2 (1 + tanh(2 d / D)).  Started on it,
    # the discrete scheme must keep it (to the O(1e-2) lattice error of a 4-site-wide
    # interface) with the interface centre fixed half-way between nodes.
    p = W.planar_2d(nx=2, ny=64, width=2.0, m=0.1)
    prm = lbm.Params(p)
    st = lbm.run(prm, lbm.init_state(prm, p["C0"]), 1000)
    C = lbm.components(prm, st.g)[1, 0, :, 0]
    y = np.arange(64)
    k = np.nonzero((C[:-1] > 0.5) & (C[1:] <= 0.5))[0][0]
    y0 = k + (C[k] - 0.5) / (C[k] - C[k + 1])
    assert abs(y0 - 47.5) < 1e-2
    ref = 0.5 * (1 + np.tanh(2 * (y0 - y) / 4.0))
    win = np.abs(y - y0) < 8
    assert np.abs(C[win] - ref[win]).max() < 1e-2
    assert abs(C.max() - 1.0) < 1e-3 and abs(C.min()) < 1e-3


@pytest.mark.slow
def test_laplace_pressure():
    # Laplace law dP = sigma / R for a 2-D droplet: the force of Eq. 34 is balanced by the
    # pressure of Eq. 38 at rest.  The diffuse interface (D = 4) makes it approximate, with an
    # error that shrinks as R grows (measured: +4.1% at R = 12, +2.5% at R = 16, 4000 steps).
    errs = []
    for R in (12.0, 16.0):
        p = W.droplet_2d(n=64, radius=R, sigma=0.01)
        prm = lbm.Params(p)
        st = lbm.run(prm, lbm.init_state(prm, p["C0"]), 4000)
        C, v, P, _ = lbm.fields(prm, st)
        dP, Reff = observables.laplace_pressure(P[0], C[1, 0])
        errs.append(abs(dP - 0.01 / Reff) / (0.01 / Reff))
        assert np.sqrt((v ** 2).sum(axis=0)).max() < 5e-5     # spurious currents only
    assert errs[0] < 0.05 and errs[1] < 0.035 and errs[1] < errs[0]


@pytest.mark.slow
def test_nonconservative_force_drifts_conservative_does_not():
    # Sec. IV A, Janus droplet: the potential form of the force (Eq. 31) makes the drop drift;
    # the conservative form (Eq. 34) keeps the mean velocity at round-off.
    p = W.janus_2d(nx=60, ny=60, radius=12, offset=15)
    prm = lbm.Params(p)
    n = 60 * 60
    cons = lbm.run(prm, lbm.init_state(prm, p["C0"]), 400)
    ncon = lbm.run(prm, lbm.init_state(prm, p["C0"]), 400, force_form="nonconservative")
    mc = np.abs(lbm.diagnostics(prm, cons)["momentum"]).max() / n
    mn = np.abs(lbm.diagnostics(prm, ncon, force_form="nonconservative")["momentum"]).max() / n
    assert mc < 1e-15
    assert mn > 1e3 * max(mc, 1e-18)


def _mode_decay_rate(tau_g, nx, steps, C0=0.1, amp=1e-4, m=0.05):
    # Decay rate of a small single-mode perturbation of a stable binary mixture (C0 outside the
    # spinodal), measured from the projection of C_0 onto cos(2 pi x / nx) at two times.
    sig = np.array([[0.0, 0.005], [0.005, 0.0]])
    p = W.base_params(9, nx, 2, 1, 2, sig, 1.0, m=m, omega_stab=0.0)
    p["tau_g"] = tau_g
    x = np.arange(nx)
    mode = np.cos(2 * np.pi * x / nx)
    C = np.zeros((2, 1, 2, nx))
    C[0] = (C0 + amp * mode)[None, None, :]
    C[1] = 1.0 - C[0]
    prm = lbm.Params(p)
    st = lbm.init_state(prm, C)
    amps, t = [], 0
    for target in steps:
        st = lbm.run(prm, st, target - t)
        t = target
        c = lbm.components(prm, st.g)[0, 0].mean(axis=0)
        amps.append(2.0 * np.mean((c - c.mean()) * mode))
    return math.log(amps[0] / amps[1]) / (steps[1] - steps[0])


@pytest.mark.slow
def test_tau_g_sets_the_mobility():
    # Eq. 43: the Cahn-Hilliard mobility is M = c_s^2 m (tau_g - 1/2).  In the linear regime a
    # mode decays at a rate proportional to M times a factor fixed by the free energy and k, so
    # the rates of tau_g = 1.4 and 0.8 are in the ratio (1.4 - 0.5) / (0.8 - 0.5) = 3, up to a
    # lattice correction of order k^2: it must shrink about fourfold when the wavelength
    # doubles, and the Richardson extrapolation of the two ratios must give 3.
    r32 = _mode_decay_rate(1.4, 32, (100, 1100)) / _mode_decay_rate(0.8, 32, (100, 1100))
    r64 = _mode_decay_rate(1.4, 64, (400, 4400)) / _mode_decay_rate(0.8, 64, (400, 4400))
    assert abs(r32 - 3.0) < 0.12
    assert abs(r64 - 3.0) < 0.3 * abs(r32 - 3.0)
    assert abs((4.0 * r64 - r32) / 3.0 - 3.0) < 0.01


def test_storage_rounding_follows_the_formats():
    # 16-bit storage of f (a reading of the paper's f: stored as f_k / w_k): the rounding is pinned
    # by values the IEEE binary16 and bfloat16 definitions fix (round to nearest, ties to even).
    r16 = lambda x: float(lbm.round_to_storage(np.array([x]), "fp16")[0])
    rbf = lambda x: float(lbm.round_to_storage(np.array([x]), "bf16")[0])
    # binary16: 11 significand bits, unit in the last place 2^-10 at 1
    assert r16(1.0 + 2.0 ** -11) == 1.0                      # tie -> even
    assert r16(1.0 + 3 * 2.0 ** -11) == 1.0 + 2.0 ** -9       # tie -> even (upwards)
    assert r16(1.0 + 2.0 ** -11 + 2.0 ** -20) == 1.0 + 2.0 ** -10
    assert r16(2049.0) == 2048.0 and r16(2051.0) == 2052.0
    assert r16(-1.0 - 3 * 2.0 ** -11) == -(1.0 + 2.0 ** -9)
    assert r16(65504.0) == 65504.0
    # bfloat16: 8 significand bits, unit in the last place 2^-7 at 1
    assert rbf(1.0 + 2.0 ** -8) == 1.0
    assert rbf(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert rbf(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7
    assert rbf(-3.0) == -3.0 and rbf(257.0) == 256.0 and rbf(259.0) == 260.0
    assert rbf(1e30) / 1e30 - 1.0 < 2.0 ** -8
    # half-unit error bounds on random values of both signs
    x = np.random.default_rng(5).uniform(-50.0, 50.0, 100000)
    assert (np.abs(lbm.round_to_storage(x, "fp16") - x) <= 2.0 ** -11 * np.abs(x)).all()
    assert (np.abs(lbm.round_to_storage(x, "bf16") - x) <= 2.0 ** -8 * np.abs(x)).all()


@pytest.mark.parametrize("q", [9, 19])
def test_store_populations_scales_by_weight_and_power_of_two(q):
    lat = lbm.Lattice(q)
    f = np.zeros((q, 1, 2, 3))
    for k in range(q):
        f[k, 0, 0, :] = lat.w[k] * 2.0 ** -10 * (1.0 + 2.0 ** -12)          # rounds down in FP16 at 2^10
        f[k, 0, 1, :] = lat.w[k] * 2.0 ** -10 * (1.0 + 3 * 2.0 ** -11)      # tie -> 1 + 2^-9
    out = lbm.store_populations(lat, f, "fp16", scale_exp=10)
    np.testing.assert_array_equal(out[0], f[0])                              # f_0 is not stored
    for k in range(1, q):
        assert (out[k, 0, 0] == lat.w[k] * 2.0 ** -10).all()
        assert (out[k, 0, 1] == lat.w[k] * 2.0 ** -10 * (1.0 + 2.0 ** -9)).all()
    # without the scale the same values sit near 2^-10 in FP16 (spacing 2^-20): barely moved
    out0 = lbm.store_populations(lat, f, "fp16", scale_exp=0)
    assert np.abs(out0[1:] - f[1:]).max() <= 2.0 ** -21 * lat.w.max()
    # BF16 ignores the scale: f_k / w_k = 2^-10 (1 + 2^-12) rounds to 2^-10
    outb = lbm.store_populations(lat, f, "bf16", scale_exp=10)
    for k in range(1, q):
        assert (outb[k, 0, 0] == lat.w[k] * 2.0 ** -10).all()
    assert lbm.store_populations(lat, f, None) is f


def test_stored_f_keeps_mass_exact_and_stays_near_full_precision():
    # With f kept in 16 bits the component populations g (full precision) still conserve mass
    # exactly, and the run stays close to the full-precision one (momentum need not be conserved).
    p = W.spinodal_2d(nx=24, ny=20)
    prm = lbm.Params(p)
    ref = lbm.run(prm, lbm.init_state(prm, p["C0"], flux_form="factored"), 40, flux_form="factored")
    C_ref = lbm.components(prm, ref.g)
    for fmt, tol in (("fp16", 1e-4), ("bf16", 2e-3)):
        st = lbm.init_state(prm, p["C0"], flux_form="factored", f_storage=fmt, scale_exp=10)
        st = lbm.run(prm, st, 40, flux_form="factored", f_storage=fmt, scale_exp=10)
        C = lbm.components(prm, st.g)
        m0 = p["C0"].reshape(prm.N, -1).sum(axis=1)
        np.testing.assert_allclose(C.reshape(prm.N, -1).sum(axis=1), m0, rtol=1e-13)
        err = np.abs(C - C_ref).max()
        assert 0 < err < tol, (fmt, err)
