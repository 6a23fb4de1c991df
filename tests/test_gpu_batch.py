"""The batched sweep against the FP64 oracle and against the single-simulation path, and its
bounded grid barrier (a wait that runs out is reported, the GPU stays usable)."""
import numpy as np
import pytest

import nfe_workloads as W
import paper_2605_22214_gb300 as nfe
from oracle import lbm

from ._lib import lib, rel

pytestmark = pytest.mark.gpu


def _mixture(nx, ny, N, seed):
    rng = np.random.default_rng(seed)
    sig = W.random_sigma(rng, N)
    C = 1.0 / N + rng.uniform(-0.05, 0.05, size=(N, 1, ny, nx))
    C /= C.sum(axis=0, keepdims=True)
    p = W.base_params(9, nx, ny, 1, N, sig, rng.uniform(0.7, 1.2, N), walls=(False, bool(seed % 2), False),
                      lambda_trt=3 / 16, m=0.05)
    p["C0"] = C
    return p


def _sims():
    return [W.lens_2d(nx=40, ny=36, radius=8), W.janus_2d(nx=48, ny=40, radius=9, offset=11),
            _mixture(33, 29, 5, 3), W.spinodal_2d(nx=64, ny=64, seed=7), _mixture(70, 45, 2, 4),
            W.droplet_2d(n=32, radius=7), _mixture(5, 7, 3, 5)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    lib()


def _single(p, steps, precision):
    with nfe.Sim(p, precision) as s:
        s.set_fields(p["C0"])
        s.step(steps)
        return s.fields()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("mode", [nfe.NFE_BATCH_PERSISTENT, nfe.NFE_BATCH_PER_STEP])
def test_batch_matches_single_simulations(precision, mode):
    sims = _sims()
    with nfe.Batch(sims, precision) as b:
        b.set_mode(mode)
        for i, p in enumerate(sims):
            b.set_fields(i, p["C0"])
        b.step(17)           # odd: parity flips
        b.step(20)
        b.sync()
        for i, p in enumerate(sims):
            Cb, vb, Pb = b.fields(i)
            Cs, vs, Ps = _single(p, 37, precision)
            tol = 1e-14 if precision == "fp64" else 1e-6
            assert np.abs(Cb - Cs).max() <= tol, i
            assert np.abs(vb - vs).max() <= tol * max(np.abs(vs).max(), 1e-30) + 1e-300, i
        info = b.info()
        assert info["nsims"] == len(sims) and info["tile_x"] == 32


def _oracle_members():
    # N = 2..5, ragged sizes (not multiples of the 32 x TY tile), walls in y on two members,
    # TRT with unequal tau, a body force, and Omega != 0 (the stabiliser of Eq. 17) on two members
    a = _mixture(37, 21, 2, 21)
    b = _mixture(45, 34, 3, 22)
    b["omega_stab"] = 1.0 / 90.0
    c = _mixture(29, 41, 4, 23)
    c["body_force"] = (2e-6, -1e-6, 0.0)
    d = _mixture(50, 19, 5, 24)
    d["omega_stab"] = 1.0 / 90.0
    e = W.lens_2d(nx=35, ny=30, radius=7)
    return [a, b, c, d, e]


@pytest.fixture(scope="module")
def oracle_members():
    sims = _oracle_members()
    out = []
    for p in sims:
        prm = lbm.Params(p)
        st = lbm.run(prm, lbm.init_state(prm, p["C0"], flux_form="factored"), 41, flux_form="factored")
        C, v, P, _ = lbm.fields(prm, st, flux_form="factored")
        out.append(dict(C=C, v=v, P=P))
    return sims, out


@pytest.mark.parametrize("precision,tol_c,tol_v", [("fp64", 1e-12, 1e-10), ("fp32", 1e-5, 1e-3)])
@pytest.mark.parametrize("mode", [nfe.NFE_BATCH_PERSISTENT, nfe.NFE_BATCH_PER_STEP])
def test_batch_members_match_oracle(oracle_members, precision, tol_c, tol_v, mode):
    # every member of one batch (its own tile code: L2-only loads, the descriptor in shared memory,
    # quartic coefficients from device memory) element by element against the FP64 oracle
    sims, ref = oracle_members
    with nfe.Batch(sims, precision) as b:
        b.set_mode(mode)
        for i, p in enumerate(sims):
            b.set_fields(i, p["C0"])
        b.step(17)
        b.step(24)
        b.sync()
        for i, o in enumerate(ref):
            Cb, vb, Pb = b.fields(i)
            errs = dict(C=rel(Cb, o["C"]), v=rel(vb, o["v"]), P=rel(Pb, o["P"]))
            assert errs["C"] <= tol_c, (i, errs)
            assert errs["v"] <= tol_v and errs["P"] <= tol_v, (i, errs)
            assert b.diagnostics(i)["step"] == 41


@pytest.mark.parametrize("precision,tol_c,tol_v", [("fp64", 1e-12, 1e-10), ("fp32", 1e-5, 1e-3)])
def test_batch_with_no_phi_and_stored_g_members_matches_oracle(precision, tol_c, tol_v):
    # a batch mixing the method as stated, the no-phi ablation and stored component populations
    # (tau_g = 0.8 and 1.3): each member against the oracle's literal form of its step
    plain = _mixture(37, 21, 3, 31)
    # the no-phi member: a lens with an absent fourth component (implicit component 0)
    lens = W.lens_2d(nx=40, ny=34, radius=8)
    sig = np.full((4, 4), 0.005)
    np.fill_diagonal(sig, 0.0)
    sig[:3, :3] = lens["sigma"]
    nophi = W.base_params(9, 40, 34, 1, 4, sig, 1.0, walls=(False, True, False), m=0.05, implicit=0)
    nophi["C0"] = np.zeros((4,) + lens["C0"].shape[1:])
    nophi["C0"][:3] = lens["C0"]
    nophi["flags"] = nfe.NFE_NO_PHI
    sg1 = _mixture(45, 30, 4, 32)
    sg1["tau_g"] = 0.8
    sg2 = _mixture(33, 41, 2, 33)
    sg2["tau_g"] = 1.3
    sims = [plain, nophi, sg1, sg2]
    steps = 30
    ref = []
    for p in sims:
        prm = lbm.Params(p)
        if p.get("flags", 0) & nfe.NFE_NO_PHI:
            st = lbm.run(prm, lbm.init_state(prm, p["C0"]), steps, with_phi=False)
            C, v, P, _ = lbm.fields(prm, st)
        else:
            st = lbm.run(prm, lbm.init_state(prm, p["C0"], flux_form="factored"), steps, flux_form="factored")
            C, v, P, _ = lbm.fields(prm, st, flux_form="factored")
        ref.append(dict(C=C, v=v, P=P))
    with nfe.Batch(sims, precision) as b:
        with pytest.raises(nfe.NfeError) as e:
            b.set_mode(nfe.NFE_BATCH_PERSISTENT)
        assert e.value.status == 7
        for i, p in enumerate(sims):
            b.set_fields(i, p["C0"])
        b.step(13)           # odd: parity flips (the stored g swap with f and C)
        b.set_fields(0, sims[0]["C0"])
        b.step(steps - 13)
        b.sync()
        info = b.info()
        assert info["form"] == nfe.NFE_BATCH_PER_STEP and info["tile_y"] == 8
        for i, o in enumerate(ref):
            if i == 0:
                continue                  # restarted above
            Cb, vb, Pb = b.fields(i)
            errs = dict(C=rel(Cb, o["C"]), v=rel(vb, o["v"]), P=rel(Pb, o["P"]))
            assert errs["C"] <= tol_c, (i, errs)
            assert errs["v"] <= tol_v and errs["P"] <= tol_v, (i, errs)
        assert np.abs(b.fields(1)[0][3]).max() > 1e-7          # the absent component nucleates


def test_set_fields_after_odd_steps_and_absent_component():
    sims = _sims()[:3]
    q = sims[0]
    N = 4
    C = np.zeros((N,) + q["C0"].shape[1:])
    C[:3] = q["C0"]
    sig = np.full((N, N), 0.005)
    np.fill_diagonal(sig, 0)
    sig[:3, :3] = q["sigma"]
    absent = W.base_params(9, 40, 36, 1, N, sig, 1.0, walls=(False, True, False), m=0.05, implicit=0)
    absent["C0"] = C
    sims.append(absent)
    with nfe.Batch(sims, "fp32") as b:
        for i, p in enumerate(sims):
            b.set_fields(i, p["C0"])
        b.step(3)                       # parity 1
        b.set_fields(1, sims[1]["C0"])  # restart one simulation mid-batch
        b.step(10)
        Cb, _, _ = b.fields(1)
        Cs, _, _ = _single(sims[1], 10, "fp32")
        assert np.abs(Cb - Cs).max() <= 1e-6
        assert (b.fields(3)[0][3] == 0.0).all()
        assert b.diagnostics(3)["step"] == 13


def test_barrier_timeout_is_reported_and_gpu_stays_usable():
    sims = _sims()[:4]
    with nfe.Batch(sims, "fp32") as b:
        for i, p in enumerate(sims):
            b.set_fields(i, p["C0"])
        b.step(2)
        b.sync()
        # the next launch's barriers wait for one CTA more than exist, with a short limit
        b.set_mode(nfe.NFE_BATCH_PERSISTENT)
        b.set_barrier_test(20000, 1)
        b.step(4)
        b.step(2)          # an ordinary launch queued behind it keeps the timeout recorded
        with pytest.raises(nfe.NfeError) as e:
            b.sync()
        assert e.value.status == 6
        b.sync()           # reported once
        # the context is still usable: reset and step normally
        for i, p in enumerate(sims):
            b.set_fields(i, p["C0"])
        b.step(5)
        b.sync()
        Cb, _, _ = b.fields(0)
        Cs, _, _ = _single(sims[0], 5, "fp32")
        assert np.abs(Cb - Cs).max() <= 1e-6
