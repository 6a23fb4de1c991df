"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: FP64 volume fractions 1e-12 relative after 100 steps, FP32 1e-5;
populations, velocity and pressure are small derived signals (their largest
value can be 1e-6 while C is O(1)), so they are compared relative to their own
largest value with 1e-10 (FP64) and 1e-3 (FP32).  An absent evolved component
must be exactly 0.0.
"""
import numpy as np
import pytest

import nfe_workloads as W
import paper_2605_22214_gb300 as nfe
from oracle import lbm, observables

from ._lib import lib, rel

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(C=1e-12, f=1e-10), "fp32": dict(C=1e-5, f=1e-3)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    lib()


def oracle_run(p, steps, force_form="conservative"):
    prm = lbm.Params(p)
    st = lbm.init_state(prm, p["C0"], flux_form="factored")
    st = lbm.run(prm, st, steps, flux_form="factored", force_form=force_form)
    C, v, P, _ = lbm.fields(prm, st, flux_form="factored", force_form=force_form)
    diag = lbm.diagnostics(prm, st, flux_form="factored", force_form=force_form)
    return dict(C=C, v=v, P=P, f=st.f[1:], diag=diag)


def gpu_run(p, steps, precision="fp64", variant=None, **kw):
    with nfe.Sim(p, precision, **kw) as s:
        s.set_fields(p["C0"])
        if variant is not None:
            s.set_variant(variant)
        s.step(steps)
        s.sync()
        C, v, P = s.fields()
        f = s.populations()
        diag = s.diagnostics()
    return dict(C=C, v=v, P=P, f=f, diag=diag)


def compare_diagnostics(dg, do, precision, n):
    """nfe_diagnostics against the oracle's global sums (the FP64 reductions of step a7).

    Mass, the force sums and the extrema are compared with the field tolerances; the momentum
    sum, a sum of n small velocities, within n times the velocity tolerance of its largest
    site value."""
    tol = TOL[precision]
    assert dg["step"] == do["step"]
    assert dg["nonfinite"] == do["nonfinite"] == 0
    np.testing.assert_allclose(dg["mass"], do["mass"], rtol=tol["C"], atol=0)
    cmax = np.abs(do["max_abs_C"]).max()
    assert np.abs(dg["max_abs_C"] - do["max_abs_C"]).max() <= tol["C"] * cmax
    assert np.abs(dg["min_C"] - do["min_C"]).max() <= tol["C"] * cmax
    fabs = do["force_abs_sum"].sum()
    np.testing.assert_allclose(dg["force_abs_sum"], do["force_abs_sum"], rtol=tol["f"], atol=tol["f"] * fabs)
    assert np.abs(dg["force_sum"] - do["force_sum"]).max() <= tol["f"] * fabs
    vmax = do["max_speed"]
    assert abs(dg["max_speed"] - vmax) <= tol["f"] * vmax + 1e-300
    assert np.abs(dg["momentum"] - do["momentum"]).max() <= tol["f"] * n * vmax + 1e-300


def compare(p, steps, precision, force_form="conservative", **kw):
    o = oracle_run(p, steps, force_form)
    if force_form == "nonconservative":
        kw["flags"] = kw.get("flags", 0) | nfe.NFE_NONCONSERVATIVE_FORCE
    g = gpu_run(p, steps, precision, **kw)
    tol = TOL[precision]
    errs = {k: rel(g[k], o[k]) for k in ("C", "f", "v", "P")}
    assert errs["C"] <= tol["C"], errs
    for k in ("f", "v", "P"):
        assert errs[k] <= tol["f"], errs
    compare_diagnostics(g["diag"], o["diag"], precision, p["nx"] * p["ny"] * p["nz"])
    return o, g, errs


def _mixture(nx, ny, N, seed, walls=(False, False, False), taus=None, lam=-1.0, fb=(0, 0, 0), omega=float("nan")):
    rng = np.random.default_rng(seed)
    sig = W.random_sigma(rng, N)
    C = 1.0 / N + rng.uniform(-0.05, 0.05, size=(N, 1, ny, nx))
    C /= C.sum(axis=0, keepdims=True)
    p = W.base_params(9, nx, ny, 1, N, sig, taus if taus is not None else 1.0, walls=walls, lambda_trt=lam,
                      m=0.05, body_force=fb, omega_stab=omega)
    p["C0"] = C
    return p


CASES = {
    "lens_walls_N3": lambda: W.lens_2d(nx=40, ny=36, radius=8),
    "spinodal_N4": lambda: W.spinodal_2d(nx=48, ny=40),
    "janus_N4": lambda: W.janus_2d(nx=48, ny=40, radius=9, offset=11),
    "mixture_N5_trt_omega_wallsx": lambda: _mixture(36, 30, 5, 11, walls=(True, False, False),
                                                    taus=[0.6, 0.8, 1.0, 0.7, 1.3], lam=3 / 16,
                                                    fb=(1e-6, -2e-6, 0), omega=1 / 90),
    "mixture_N8": lambda: _mixture(20, 18, 8, 12),
    "janus3d_N4": lambda: W.janus_3d(n=16, radius=4),
    "poiseuille3d_N7": lambda: W.layered_poiseuille(nx=6, ny=5, nz=24),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_fp64_parity_100_steps(case):
    compare(CASES[case](), 100, "fp64")


@pytest.mark.parametrize("case", ["lens_walls_N3", "spinodal_N4", "janus3d_N4", "poiseuille3d_N7"])
def test_fp32_parity_100_steps(case):
    compare(CASES[case](), 100, "fp32")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["janus_N4", "mixture_N5_trt_omega_wallsx", "janus3d_N4", "d3q19_walls_N4"])
def test_nonconservative_force_parity_100_steps(case, precision):
    # The non-conservative surface-tension force of Eq. 31 (F_s = sum_i mu_i grad C_i, the
    # paper's negative control, NFE_NONCONSERVATIVE_FORCE) on D2Q9 and D3Q19 against the oracle's
    # literal Eq. 31 with the chemical potentials of Eq. 7.
    p = _mixture3d(19, 13, 14, 4, 51, (True, False, True)) if case == "d3q19_walls_N4" else CASES[case]()
    compare(p, 100, precision, force_form="nonconservative")


@pytest.mark.parametrize("shape,walls,N", [((3, 5), (False, True), 2), ((5, 1), (False, False), 3),
                                           ((3, 4), (True, False), 2), ((7, 3), (True, True), 4)])
def test_tiny_and_degenerate_grids(shape, walls, N):
    nx, ny = shape
    p = _mixture(nx, ny, N, 20 + nx, walls=(walls[0], walls[1], False))
    compare(p, 30, "fp64")


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_full_size_spinodal_elementwise(precision):
    # The benchmarked workload (512 x 512, N = 4) element by element after 3 steps.
    p = W.spinodal_2d()
    compare(p, 3, precision)


def _absent_lens(N=4):
    p = W.lens_2d(nx=40, ny=36, radius=8)
    C = np.zeros((N,) + p["C0"].shape[1:])
    C[:3] = p["C0"]
    sig = np.full((N, N), 0.005)
    np.fill_diagonal(sig, 0)
    sig[:3, :3] = p["sigma"]
    q = W.base_params(9, 40, 36, 1, N, sig, 1.0, walls=(False, True, False), m=0.05, implicit=0)
    q["C0"] = C
    return q


@pytest.mark.parametrize("precision", ["fp64", "fp32", "f16", "bf16"])
def test_absent_component_stays_exactly_zero(precision):
    p = _absent_lens()
    with nfe.Sim(p, precision, scale_exp=10) as s:
        s.set_fields(p["C0"])
        for _ in range(3):
            s.step(100)
            C, _, _ = s.fields()
            assert (C[3] == 0.0).all()
    p = W.layered_poiseuille(nx=6, ny=5, nz=24)
    with nfe.Sim(p, precision, scale_exp=10) as s:
        s.set_fields(p["C0"])
        s.step(300)
        C, _, _ = s.fields()
        assert (C[6] == 0.0).all()


@pytest.mark.parametrize("precision,tol_c,tol_v", [("fp64", 1e-12, 1e-10), ("fp32", 1e-5, 1e-3)])
def test_no_phi_ablation_matches_oracle_and_nucleates(precision, tol_c, tol_v):
    # The no-phi ablation (Eq. 12 without phi_j, the paper's negative control): the GPU follows
    # the oracle's literal flux potential without phi_j, and the absent fourth component appears
    # at the interfaces (with phi_j it stays exactly zero: test_absent_component_stays_exactly_zero).
    p = _absent_lens()
    steps = 60
    prm = lbm.Params(p)
    st = lbm.run(prm, lbm.init_state(prm, p["C0"]), steps, with_phi=False)
    Co, vo, Po, _ = lbm.fields(prm, st)
    g = gpu_run(p, steps, precision, flags=nfe.NFE_NO_PHI)
    assert rel(g["C"], Co) < tol_c
    assert rel(g["v"], vo) < tol_v
    assert np.abs(Co[3]).max() > 1e-6 and np.abs(g["C"][3]).max() > 1e-6
    if precision == "fp64":
        assert rel(g["C"][3], Co[3]) < 1e-9


@pytest.mark.parametrize("precision,tol_c,tol_v", [("fp64", 1e-12, 1e-10), ("fp32", 1e-5, 1e-3)])
def test_no_phi_ablation_d3q19_matches_oracle_and_nucleates(precision, tol_c, tol_v):
    # The no-phi ablation on D3Q19 (split form of the step): a 3-D lens-like layout with an absent
    # fourth component, against the oracle's literal Eq. 12 without phi_j; the absent component
    # appears where three present ones meet.
    n = 24
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    below = W.tanh_step(n / 2 - 0.5 - z)
    drop = W.tanh_step(6.0 - np.sqrt((x - n / 2 + 0.5) ** 2 + (y - n / 2 + 0.5) ** 2 + (z - n / 2 + 0.5) ** 2))
    C = np.zeros((4, n, n, n))
    C[0] = below * (1 - drop)
    C[1] = (1 - below) * (1 - drop)
    C[2] = drop
    sig = np.full((4, 4), 0.005)
    np.fill_diagonal(sig, 0)
    sig[0, 1] = sig[1, 0] = 0.01
    sig[0, 2] = sig[2, 0] = sig[1, 2] = sig[2, 1] = 0.008
    p = W.base_params(19, n, n, n, 4, sig, 1.0, walls=(False, False, True), m=0.05, implicit=0)
    p["C0"] = C
    steps = 40
    prm = lbm.Params(p)
    st = lbm.run(prm, lbm.init_state(prm, p["C0"]), steps, with_phi=False)
    Co, vo, Po, _ = lbm.fields(prm, st)
    g = gpu_run(p, steps, precision, flags=nfe.NFE_NO_PHI)
    assert rel(g["C"], Co) < tol_c
    assert rel(g["v"], vo) < tol_v
    assert np.abs(Co[3]).max() > 1e-7 and np.abs(g["C"][3]).max() > 1e-7
    if precision == "fp64":
        assert rel(g["C"][3], Co[3]) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case,tau_g", [("lens_walls_N3", 0.8), ("spinodal_N4", 1.3)])
def test_stored_g_tau_g_parity_with_oracle(precision, case, tau_g):
    # tau_g != 1 (Sec. III B): the component populations are stored, relaxed with 1/tau_g,
    # pulled and bounced back; the GPU follows the oracle's literal g populations.
    p = CASES[case]()
    p["tau_g"] = tau_g
    compare(p, 100, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("tau_g,walls", [(0.8, (False, True, True)), (1.3, (True, False, False))])
def test_stored_g_tau_g_d3q19_parity_with_oracle(precision, tau_g, walls):
    # tau_g != 1 on D3Q19 (split form of the step, the stored g pulled, relaxed and bounced back
    # in the gather kernel) against the oracle's literal g populations
    p = _mixture3d(21, 13, 14, 4, 60, walls)
    p["tau_g"] = tau_g
    compare(p, 60, precision)


def test_stored_g_conservation_checkpoint_and_absent_component():
    # tau_g = 1.3, FP64: per-component mass to round-off, a checkpoint (which carries g)
    # restores the run bitwise, and an absent component stays exactly zero.
    p = W.spinodal_2d(nx=48, ny=40, seed=7)
    p["tau_g"] = 1.3
    with nfe.Sim(p, "fp64") as s:
        s.set_fields(p["C0"])
        m0 = s.diagnostics()["mass"]
        s.step(50)
        snap = s.get_state()
        s.step(50)
        a = s.get_state()
        np.testing.assert_allclose(s.diagnostics()["mass"], m0, rtol=1e-12)
        s.set_state(snap)
        s.step(50)
        assert np.array_equal(s.get_state(), a)
    q = _absent_lens()
    q["tau_g"] = 1.3
    with nfe.Sim(q, "fp64") as s:
        s.set_fields(q["C0"])
        s.step(200)
        C, _, _ = s.fields()
        assert (C[3] == 0.0).all()


def test_mass_and_momentum_conservation_fp64():
    p = W.janus_2d(nx=64, ny=64, radius=12, offset=15)
    with nfe.Sim(p, "fp64") as s:
        s.set_fields(p["C0"])
        d0 = s.diagnostics()
        for _ in range(5):
            s.step(200)
            d = s.diagnostics()
            np.testing.assert_allclose(d["mass"], d0["mass"], rtol=1e-13)
            assert np.abs(d["force_sum"]).max() <= 1e-13 * d["force_abs_sum"].sum()
            assert np.abs(d["momentum"]).max() <= 1e-13 * d["force_abs_sum"].sum() + 1e-16
            assert d["nonfinite"] == 0


def test_momentum_changes_by_body_force():
    p = W.janus_2d(nx=48, ny=48, radius=9, offset=11)
    p["body_force"] = (1e-6, -5e-7, 0.0)
    n = 48 * 48
    with nfe.Sim(p, "fp64") as s:
        s.set_fields(p["C0"])
        s.step(10)
        m0 = s.diagnostics()["momentum"]
        s.step(50)
        m1 = s.diagnostics()["momentum"]
    np.testing.assert_allclose(m1 - m0, 50 * n * np.array(p["body_force"]), rtol=1e-10, atol=1e-16)


def test_checkpoint_roundtrip_and_graph_replay_are_bitwise():
    p = W.spinodal_2d(nx=40, ny=32, seed=3)
    with nfe.Sim(p, "fp32") as s:
        s.set_fields(p["C0"])
        s.step(5)
        snap = s.get_state()
        s.step(11)                # graph replay (5 x 2 steps) + one direct step
        a = s.get_state()
        s.set_state(snap)
        for _ in range(11):
            s.step(1)             # direct launches only
        b = s.get_state()
        s.set_state(snap)
        s.profile_enable(True)
        s.step(11)                # timed launches
        c = s.get_state()
        prof = s.profile_read()
    assert np.array_equal(a, b) and np.array_equal(a, c)
    assert set(prof) == {"fused_step"}
    assert prof["fused_step"][0] == 11


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_tile_variants_are_bitwise_identical(precision):
    # every tile shape of the fused D2Q9 step computes each site the same way
    for p in (W.lens_2d(nx=70, ny=45, radius=9), W.spinodal_2d(nx=33, ny=29, seed=8)):
        states = []
        with nfe.Sim(p, precision) as s:
            nv = s.info()["nvariants"]
            assert nv == 3
            for v in range(nv):
                s.set_fields(p["C0"])
                s.set_variant(v)
                s.step(25)
                states.append(s.get_state())
        for st in states[1:]:
            assert np.array_equal(st, states[0])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("lattice", [9, 19])
def test_component_force_matches_oracle(precision, lattice):
    # a body force acting on one component in proportion to its volume fraction (F += C_c F_c)
    if lattice == 9:
        p = W.janus_2d(nx=48, ny=40, radius=9, offset=11)
        p["component_force"] = (3e-6, -2e-6, 0.0)
    else:
        p = _mixture3d(21, 13, 18, 3, 31, (False, True, False))
        p["component_force"] = (1e-6, 2e-6, -3e-6)
    p["component_force_index"] = 1
    compare(p, 40, precision)


def _mixture3d(nx, ny, nz, N, seed, walls):
    rng = np.random.default_rng(seed)
    sig = W.random_sigma(rng, N)
    C = 1.0 / N + rng.uniform(-0.05, 0.05, size=(N, nz, ny, nx))
    C /= C.sum(axis=0, keepdims=True)
    p = W.base_params(19, nx, ny, nz, N, sig, rng.uniform(0.7, 1.2, N), walls=walls, lambda_trt=3 / 16,
                      m=0.05, body_force=(1e-6, 0, -2e-6))
    p["C0"] = C
    return p


@pytest.mark.parametrize("shape,walls,N", [((20, 13, 17), (False, False, True), 3),
                                           ((5, 3, 4), (False, False, False), 2),
                                           ((35, 9, 10), (True, True, False), 4),
                                           ((6, 7, 12), (True, False, True), 5)])
def test_d3q19_ragged_and_walls_fp64(shape, walls, N):
    nx, ny, nz = shape
    compare(_mixture3d(nx, ny, nz, N, 40 + N, walls), 25, "fp64")


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("case", ["walls_yz_N4", "periodic_N5_omega"])
def test_d3q19_variants_are_bitwise_identical(precision, case):
    # the fused step (32x4, 32x8) and the split step (physics + gather kernels, 32x8, 32x4)
    # compute every site with the same arithmetic
    if case == "walls_yz_N4":
        p = _mixture3d(37, 11, 19, 4, 9, (False, True, True))
    else:
        p = _mixture3d(33, 21, 17, 5, 10, (False, False, False))
        p["omega_stab"] = 1.0 / 90.0
    states = []
    with nfe.Sim(p, precision) as s:
        nv = s.info()["nvariants"]
        assert nv == 4
        for v in range(nv):
            s.set_fields(p["C0"])
            s.set_variant(v)
            s.step(13)
            # the fused form exists for N <= 4; above, variants 0 and 1 alias the split ones
            assert s.info()["kernels_per_step"] == (2 if v >= 2 or p["N"] > 4 else 1)
            states.append(s.get_state())
    for st in states[1:]:
        assert np.array_equal(st, states[0])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("variant", [2, 3])
def test_d3q19_split_step_parity_with_oracle(precision, variant):
    # the split D3Q19 step (v and S through HBM) against the oracle directly, with walls and TRT
    compare(_mixture3d(35, 9, 10, 4, 44, (True, True, False)), 40, precision, variant=variant)


def test_nonfinite_flag_reported():
    p = W.spinodal_2d(nx=16, ny=16, seed=4)
    C0 = p["C0"].copy()
    C0[1, 0, 3, 4] = np.nan
    with nfe.Sim(p, "fp64") as s:
        s.set_fields(C0)
        s.step(2)
        with pytest.raises(nfe.NfeError) as e:
            s.sync()
        assert e.value.status == 5
        assert s.diagnostics()["nonfinite"] == 1


@pytest.mark.parametrize("lattice", ["d2q9", "d3q19"])
@pytest.mark.parametrize("precision,fmt", [("f16", "fp16"), ("bf16", "bf16")])
def test_low_precision_storage_matches_oracle_with_stored_f(precision, fmt, lattice):
    # 16-bit storage of f against the oracle stepping in FP64 with f kept in the same format
    # after every step (f_k / w_k, times 2^10 for FP16).  After a few steps nearly every stored
    # value within four binades of the largest is the one that oracle stores (a value differs
    # only where the FP32 and FP64 arithmetic straddle a rounding boundary, and then by one
    # unit); the full-precision oracle's f, put through the same rounding, differs in far more
    # of them.  (Smaller values come out of cancelling terms, where the FP32 rounding error
    # reaches the 16-bit unit.)  Over many steps the one-unit differences spread through v into
    # C, so the longer run checks C against a bound scaled by the format's unit (measured: FP16
    # 8.5e-6 and 7.4e-7, BF16 5.1e-5 and 5.1e-6 for D2Q9 200 and D3Q19 60 steps).
    if lattice == "d2q9":
        p, long_steps = W.janus_2d(nx=48, ny=48, radius=8.0, offset=12.0), 200
    else:
        p, long_steps = W.janus_3d(n=32, radius=4.0), 60
    prm = lbm.Params(p)
    sc = 2.0 ** 10 if fmt == "fp16" else 1.0
    w = prm.lat.w[1:].reshape((-1,) + (1,) * (p["C0"].ndim - 1))

    def stored(f):          # the 16-bit value a population is kept as, read back
        return lbm.round_to_storage(np.asarray(f) / w * sc, fmt)

    steps = 4
    st = lbm.init_state(prm, p["C0"], flux_form="factored", f_storage=fmt, scale_exp=10)
    st = lbm.run(prm, st, steps, flux_form="factored", f_storage=fmt, scale_exp=10)
    o_plain = oracle_run(p, steps)
    g = gpu_run(p, steps, precision, scale_exp=10)
    h_gpu, h_emul, h_plain = stored(g["f"]), stored(st.f[1:]), stored(o_plain["f"])
    big = np.abs(h_emul) >= np.abs(h_emul).max() / 16
    m_emul = float(np.mean(h_gpu[big] != h_emul[big]))
    m_plain = float(np.mean(h_gpu[big] != h_plain[big]))
    print(f"{lattice} {precision}: stored f after {steps} steps ({big.mean():.2f} of the values within four binades "
          f"of the largest) differs from the stored-f oracle in {m_emul:.2e} of them, from the rounded "
          f"full-precision oracle in {m_plain:.2e}; all values {np.mean(h_gpu != h_emul):.2e} / "
          f"{np.mean(h_gpu != h_plain):.2e}")
    assert m_emul < 0.02, m_emul
    assert m_emul < 0.2 * m_plain, (m_emul, m_plain)
    st = lbm.init_state(prm, p["C0"], flux_form="factored", f_storage=fmt, scale_exp=10)
    st = lbm.run(prm, st, long_steps, flux_form="factored", f_storage=fmt, scale_exp=10)
    g = gpu_run(p, long_steps, precision, scale_exp=10)
    e = rel(g["C"], lbm.components(prm, st.g))
    print(f"{lattice} {precision}: C after {long_steps} steps vs the stored-f oracle {e:.3e}")
    assert e < {"fp16": 5e-5, "bf16": 5e-4}[fmt], e


@pytest.mark.parametrize("precision", ["f16", "bf16"])
def test_low_precision_storage_tracks_fp32(precision):
    # FP16/BF16 storage of f as deviations f_k / w_k: C stays close to the FP32 run.
    p = W.spinodal_2d(nx=48, ny=40)
    g32 = gpu_run(p, 200, "fp32")
    glo = gpu_run(p, 200, precision, scale_exp=10)
    assert rel(glo["C"], g32["C"]) < (1e-4 if precision == "f16" else 1e-3)
