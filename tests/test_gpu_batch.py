"""The batched persistent kernel against the single-simulation path, and its
bounded grid barrier (a wait that runs out is reported, the GPU stays usable)."""
import numpy as np
import pytest

import nfe_workloads as W
import paper_2605_22214_gb300 as nfe

from ._lib import lib

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
        with pytest.raises(nfe.NfeError) as e:
            b.sync()
        assert e.value.status == 6
        # the context is still usable: reset and step normally
        for i, p in enumerate(sims):
            b.set_fields(i, p["C0"])
        b.step(5)
        b.sync()
        Cb, _, _ = b.fields(0)
        Cs, _, _ = _single(sims[0], 5, "fp32")
        assert np.abs(Cb - Cs).max() <= 1e-6
