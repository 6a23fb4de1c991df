"""Open and complex boundaries on the GPU (nfe_set_geometry) against the oracle's
oracle/boundaries.py on the same seeded inputs: solid nodes, inlets and the convective
outflow, at a small ragged size (several 32 x 8 tiles, ragged in x and y) and at the full
emulsion layout, plus checkpoints and the validation of the entry point.

Tolerances as in the other parity tests: volume fractions 1e-12 (FP64) / 1e-5 (FP32)
relative to their largest value; populations, velocity and pressure 1e-10 / 1e-3 relative to
their own largest value."""
import numpy as np
import pytest

import nfe_workloads as W
import paper_2605_22214_gb300 as nfe
from oracle import boundaries as B
from oracle import lbm

from ._lib import lib, rel

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(C=1e-12, f=1e-10), "fp32": dict(C=1e-5, f=1e-3)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    lib()


def oracle_run(p, steps):
    prm = lbm.Params(p)
    g = p["geometry"]
    geo = B.Geometry(prm, g["node"], g["inlets"], g["outflow"])
    st = B.init_state(prm, geo, p["C0"], flux_form="factored")
    st = B.run(prm, geo, st, steps, flux_form="factored")
    C, v, P, _ = B.fields(prm, geo, st, flux_form="factored")
    return dict(C=C, v=v, P=P, f=st.f[1:], geo=geo)


def gpu_run(p, steps, precision, geometry_first=False):
    g = p["geometry"]
    with nfe.Sim(p, precision) as s:
        if geometry_first:
            s.set_geometry(g["node"], g["inlets"], g["outflow"])
            s.set_fields(p["C0"])
        else:
            s.set_fields(p["C0"])
            s.set_geometry(g["node"], g["inlets"], g["outflow"])
        s.step(steps)
        s.sync()
        C, v, P = s.fields()
        f = s.populations()
        state = s.get_state()
    return dict(C=C, v=v, P=P, f=f, state=state)


def _check(o, g, precision):
    tol = TOL[precision]
    fl = o["geo"].fluid
    errs = dict(C=rel(g["C"], o["C"]), v=rel(g["v"], o["v"]), P=rel(g["P"], o["P"]),
                f=rel(g["f"][:, fl], o["f"][:, fl]))
    assert errs["C"] <= tol["C"], errs
    for k in ("v", "P", "f"):
        assert errs[k] <= tol["f"], errs
    return errs


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("outflow", [True, False])
def test_open_channel_matches_oracle(precision, outflow):
    p = W.open_channel_2d(70, 36, 3, outflow=outflow)
    steps = 40
    _check(oracle_run(p, steps), gpu_run(p, steps, precision), precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_porous_channel_matches_oracle(precision):
    # the bench's porous-channel layout (posts every 16 sites, inlet column, outflow) at 130 x 44
    p = W.porous_channel_2d(nx=130, ny=44)
    steps = 25
    _check(oracle_run(p, steps), gpu_run(p, steps, precision), precision)


def test_geometry_and_fields_in_either_order():
    p = W.open_channel_2d(70, 36, 3)
    a = gpu_run(p, 10, "fp64")
    b = gpu_run(p, 10, "fp64", geometry_first=True)
    assert np.array_equal(a["state"], b["state"])


def test_emulsion_layout_matches_oracle_at_full_size():
    # the 600 x 140 emulsion generator in the launch configuration the benchmark times
    p = W.emulsion_2d()
    steps = 12
    o = oracle_run(p, steps)
    for precision in ("fp64", "fp32"):
        _check(o, gpu_run(p, steps, precision), precision)


def test_pals_layout_matches_oracle_at_full_size():
    # the 400 x 140 patterned liquid surface: edge walls, solid posts, a body force on fluid 2
    p = W.pals_2d()
    steps = 10
    o = oracle_run(p, steps)
    for precision in ("fp64", "fp32"):
        _check(o, gpu_run(p, steps, precision), precision)


def test_pals_droplet_moves_with_the_force_on_it():
    # centre-of-mass velocity of fluid 2, int C_2 v_x / int C_2 (Sec. V): pushed along +x by the
    # force on fluid 2, far above the residual velocity of the same layout without the force
    def vcm(force):
        p = W.pals_2d(force=force)
        g = p["geometry"]
        with nfe.Sim(p, "fp32") as s:
            s.set_fields(p["C0"])
            s.set_geometry(g["node"], g["inlets"], g["outflow"])
            s.step(3000)
            s.sync()
            C, v, _ = s.fields()
        return float((C[1] * v[0]).sum() / C[1].sum())
    moved, rest = vcm(3e-7), vcm(0.0)
    assert moved > 0 and moved > 20 * abs(rest)


def test_geometry_checkpoint_restores_bit_for_bit():
    p = W.open_channel_2d(70, 36, 4)
    g = p["geometry"]
    with nfe.Sim(p, "fp32") as s:
        s.set_fields(p["C0"])
        s.set_geometry(g["node"], g["inlets"], g["outflow"])
        info = s.info()
        plain = 8 + 8 * s.n * 4 + 3 * s.n * 4
        assert info["state_bytes"] == plain + 3 * 36 * 4          # + the ghost column
        s.step(7)
        snap = s.get_state()
        s.step(9)
        ref = s.get_state()
        s.set_state(snap)
        s.step(9)
        assert np.array_equal(s.get_state(), ref)
        s.set_geometry(None)
        assert s.info()["state_bytes"] == plain


def test_inflow_fills_the_channel_and_solid_nodes_stay_put():
    # 1500 steps of the emulsion generator: the inlet fluids enter, nothing goes non-finite,
    # and solid and inlet nodes keep their state bit for bit
    p = W.emulsion_2d()
    g = p["geometry"]
    node = g["node"]
    with nfe.Sim(p, "fp32") as s:
        s.set_fields(p["C0"])
        s.set_geometry(node, g["inlets"], g["outflow"])
        C0, _, _ = s.fields()
        f0 = s.populations()
        s.step(1500)
        s.sync()
        C1, v1, _ = s.fields()
        f1 = s.populations()
    fl = node == W.FLUID
    assert C1[1][fl].sum() > C0[1][fl].sum() + 10.0            # fluid 2 came in through its inlets
    assert np.array_equal(C1[:, ~fl], C0[:, ~fl])
    assert np.array_equal(f1[:, ~fl], f0[:, ~fl])
    assert np.abs(v1[:, node == W.SOLID]).max() == 0.0
    assert np.isfinite(C1).all() and np.abs(v1).max() < 0.1


def test_geometry_validation():
    p = W.open_channel_2d(40, 20, 3)
    g = p["geometry"]
    with nfe.Sim(p, "fp64") as s:
        bad = g["node"].copy()
        bad[0, 5, 5] = 9                                          # class without an inlet row
        with pytest.raises(nfe.NfeError):
            s.set_geometry(bad, g["inlets"], True)
        rows = g["inlets"].copy()
        rows[0, 2] += 0.1                                         # C_b no longer sums to 1
        with pytest.raises(nfe.NfeError):
            s.set_geometry(g["node"], rows, True)
        open_left = g["node"].copy()
        open_left[0, 5, 0] = W.FLUID                              # fluid on the inflow edge
        with pytest.raises(nfe.NfeError):
            s.set_geometry(open_left, g["inlets"], True)
        s.set_geometry(open_left, g["inlets"], False)             # fine without the outflow
    q = W.janus_3d(n=16, radius=4.0)
    with nfe.Sim(q, "fp32") as s:
        s.set_geometry(np.zeros(16 ** 3, np.uint8))              # D3Q19: every boundary kind
        with pytest.raises(nfe.NfeError) as e:                   # fluid in the inflow plane x = 0
            s.set_geometry(np.zeros(16 ** 3, np.uint8), outflow=True)
        assert e.value.status == 1
        one = np.zeros((1, 3 + q["N"]))                          # D3Q19 rows: v_b (3), C_b (N)
        one[0, 3] = 1.0
        node = np.zeros(16 ** 3, np.uint8)
        node[0] = W.INLET0
        s.set_geometry(node, one)
        one[0, 4] = 0.5                                           # C_b no longer sums to 1
        with pytest.raises(nfe.NfeError) as e:
            s.set_geometry(node, one)
        assert e.value.status == 1
    r = dict(p, tau_g=1.3)
    with nfe.Sim(r, "fp64") as s:
        with pytest.raises(nfe.NfeError) as e:
            s.set_geometry(g["node"], g["inlets"], True)
        assert e.value.status == 7


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_porous_3d_matches_oracle(precision):
    # D3Q19 with solid cubes, a slab with a window, walls in z and a body force along x, on a
    # grid ragged against the tiles in x and y
    p = W.porous_3d()
    steps = 30
    _check(oracle_run(p, steps), gpu_run(p, steps, precision), precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
def test_d3q19_solid_layers_equal_edge_walls_bitwise(precision):
    # the same box bounded by edge walls in y and z, and by solid layers around it (periodic
    # there): solid links take exactly the wall rules, so the interior states agree bit for bit
    nx, ny, nz, N = 40, 18, 12, 4
    a = W.porous_3d(nx, ny, nz, N, walls=(False, True, True))
    b = W.porous_3d(nx, ny + 2, nz + 2, N, walls=(False, False, False))
    node = np.zeros((nz + 2, ny + 2, nx), np.uint8)
    node[0] = node[-1] = W.SOLID
    node[:, 0] = node[:, -1] = W.SOLID
    node[1:-1, 1:-1] = a["geometry"]["node"]
    C = np.zeros((N, nz + 2, ny + 2, nx))
    C[0] = 1.0
    C[:, 1:-1, 1:-1] = a["C0"]
    b = dict(b, sigma=a["sigma"], C0=C)
    b["geometry"] = dict(node=node, inlets=np.zeros((0, 2 + N)), outflow=False)
    ga, gb = gpu_run(a, 25, precision), gpu_run(b, 25, precision)
    np.testing.assert_array_equal(gb["f"][:, 1:-1, 1:-1], ga["f"])
    np.testing.assert_array_equal(gb["C"][:, 1:-1, 1:-1], ga["C"])
    assert np.abs(gb["v"][:, node == W.SOLID]).max() == 0.0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("outflow", [False, True])
def test_inlet_channel_3d_matches_oracle(precision, outflow):
    # D3Q19 inlets (two in the x = 0 plane, one in a wall plane), solid planes and a post, with
    # and without the convective outflow on the plane x = nx - 1
    p = W.inlet_channel_3d(outflow=outflow)
    steps = 30
    o, g = oracle_run(p, steps), gpu_run(p, steps, precision)
    _check(o, g, precision)
    if outflow:
        # the checkpoint holds the ghost column: a restored state steps on bit for bit
        with nfe.Sim(p, precision) as s:
            s.set_fields(p["C0"])
            s.set_geometry(p["geometry"]["node"], p["geometry"]["inlets"], True)
            s.set_state(g["state"])
            s.step(5)
            s.sync()
            a = s.get_state()
        with nfe.Sim(p, precision) as s:
            s.set_fields(p["C0"])
            s.set_geometry(p["geometry"]["node"], p["geometry"]["inlets"], True)
            s.step(steps + 5)
            s.sync()
            b = s.get_state()
        assert np.array_equal(a[8:], b[8:])


def test_uniform_inflow_is_a_fixed_point_d3q19_gpu():
    # the oracle's pin on the GPU: a uniform mixture moving at v_b, fed by an inlet plane holding
    # the same state, periodic in x, stays as it is
    N, nx, ny, nz = 3, 40, 10, 8
    sig = np.array([[0.0, 0.006, 0.007], [0.006, 0.0, 0.005], [0.007, 0.005, 0.0]])
    p = W.base_params(W.D3Q19, nx, ny, nz, N, sig, 0.8, omega_stab=1 / 90)
    node = np.zeros((nz, ny, nx), np.uint8)
    node[..., 0] = W.INLET0
    Cb, vb = np.array([0.2, 0.5, 0.3]), (0.01, 0.003, -0.004)
    C0 = np.broadcast_to(Cb[:, None, None, None], (N, nz, ny, nx)).copy()
    v0 = np.zeros((3, nz, ny, nx))
    v0[0], v0[1], v0[2] = vb
    with nfe.Sim(p, "fp64") as s:
        s.set_fields(C0, v0)
        s.set_geometry(node, np.array([[*vb, *Cb]]))
        f0 = s.populations()
        s.step(15)
        s.sync()
        C, v, _ = s.fields()
        f1 = s.populations()
    fl = node == W.FLUID
    assert np.abs(f1 - f0)[:, fl].max() < 1e-15
    assert np.abs(C - C0).max() < 1e-14
    np.testing.assert_allclose(v[:, fl], np.array(vb)[:, None] * np.ones((1, int(fl.sum()))), rtol=0, atol=1e-15)
