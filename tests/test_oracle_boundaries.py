"""The oracle's open and complex boundaries (Sec. III C; oracle/boundaries.py) against what
fixes them independently of its own code: the edge walls already pinned elsewhere, exact
conservation, the closed-form plane Couette profile of a halfway bounce-back channel with a
moving wall, the fixed point of a uniform inflow, and the direction of the convective outflow."""
import numpy as np
import pytest

import nfe_workloads as W
from oracle import boundaries as B
from oracle import lbm


def _sigma3():
    return np.array([[0.0, 0.006, 0.007], [0.006, 0.0, 0.005], [0.007, 0.005, 0.0]])


def _mixture(nx, ny, seed):
    # smooth three-component field (two overlapping tanh discs), no RNG inside the method
    x, y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    rng = np.random.default_rng(seed)
    cx, cy = rng.uniform(2, nx - 2, 2), rng.uniform(2, ny - 2, 2)
    a = W.tanh_step(3.0 - np.hypot(x - cx[0], y - cy[0]))
    b = (1 - a) * W.tanh_step(2.5 - np.hypot(x - cx[1], y - cy[1]))
    return np.stack([1 - a - b, a, b])[:, None]


def test_solid_rows_are_the_edge_walls():
    # a channel bounded by edge walls (Eqs. 44-45 and the gradient rule at the domain edge)
    # and the same channel with one solid row above and below, periodic in y
    nx, ny = 10, 8
    C = _mixture(nx, ny, 3)
    pa = W.base_params(W.D2Q9, nx, ny, 1, 3, _sigma3(), 0.8, walls=(False, True, False), omega_stab=1 / 90)
    pb = W.base_params(W.D2Q9, nx, ny + 2, 1, 3, _sigma3(), 0.8, omega_stab=1 / 90)
    prm_a, prm_b = lbm.Params(pa), lbm.Params(pb)
    node = np.zeros((1, ny + 2, nx), int)
    node[:, 0] = node[:, -1] = B.SOLID
    geo = B.Geometry(prm_b, node)
    Cb = np.concatenate([C[:, :, :1], C, C[:, :, -1:]], axis=2)
    sa = lbm.run(prm_a, lbm.init_state(prm_a, C), 15)
    sb = B.run(prm_b, geo, B.init_state(prm_b, geo, Cb), 15)
    np.testing.assert_allclose(sb.f[:, :, 1:-1], sa.f, rtol=0, atol=1e-15)
    np.testing.assert_allclose(sb.g[:, :, :, 1:-1], sa.g, rtol=0, atol=1e-15)


def test_interior_post_conserves_every_component():
    nx, ny = 16, 12
    p = W.base_params(W.D2Q9, nx, ny, 1, 3, _sigma3(), 0.7, omega_stab=1 / 90)
    prm = lbm.Params(p)
    node = np.zeros((1, ny, nx), int)
    node[:, 4:8, 6:9] = B.SOLID
    geo = B.Geometry(prm, node)
    st = B.init_state(prm, geo, _mixture(nx, ny, 5))
    C0, _, _, _ = B.fields(prm, geo, st)
    st = B.run(prm, geo, st, 30)
    C1, v, _, _ = B.fields(prm, geo, st)
    m0, m1 = C0[:, geo.fluid].sum(axis=1), C1[:, geo.fluid].sum(axis=1)
    np.testing.assert_allclose(m1, m0, rtol=0, atol=1e-12 * nx * ny)
    assert np.abs(v[:, ~geo.fluid]).max() == 0.0
    assert np.abs(v[:, geo.fluid]).max() > 1e-9          # the mixture does move


def test_moving_lid_gives_the_plane_couette_profile():
    # bottom row solid, top row an inlet moving at (u, 0) with the fluid's own composition:
    # halfway walls at y = 1/2 and y = H + 1/2, so v_x(y) = u (y - 1/2) / H exactly at steady state
    H, u = 6, 0.01
    sig = np.array([[0.0, 0.005], [0.005, 0.0]])
    p = W.base_params(W.D2Q9, 3, H + 2, 1, 2, sig, 1.0)
    prm = lbm.Params(p)
    node = np.zeros((1, H + 2, 3), int)
    node[:, 0] = B.SOLID
    node[:, -1] = B.INLET0
    geo = B.Geometry(prm, node, [[u, 0.0, 1.0, 0.0]])
    C = np.zeros((2, 1, H + 2, 3))
    C[0] = 1.0
    st = B.run(prm, geo, B.init_state(prm, geo, C), 900)
    _, v, _, _ = B.fields(prm, geo, st)
    y = np.arange(1, H + 1)
    exact = u * (y - 0.5) / H
    np.testing.assert_allclose(v[0, 0, 1:-1, :], np.repeat(exact[:, None], 3, axis=1), rtol=0, atol=1e-9 * u)
    assert np.abs(v[1, 0, 1:-1]).max() < 1e-14


def test_uniform_inflow_through_to_the_outflow_is_a_fixed_point():
    # a uniform mixture flowing at v_b everywhere, fed by an inlet column holding the same state
    # and leaving through the convective outflow, stays as it is: the velocity rule's sign, the
    # inlet equilibrium (v_b and S_b of the non-pure C_b) and the outflow's weights all take part
    N, nx, ny = 3, 12, 6
    p = W.base_params(W.D2Q9, nx, ny, 1, N, _sigma3(), 0.8, omega_stab=1 / 90)
    prm = lbm.Params(p)
    node = np.zeros((1, ny, nx), int)
    node[..., 0] = B.INLET0
    Cb, vb = np.array([0.2, 0.5, 0.3]), (0.01, 0.003)
    geo = B.Geometry(prm, node, [[*vb, *Cb]], outflow=True)
    assert np.abs(geo.inlets[0][2]).max() > 0.05            # S_b of this C_b is far from 0
    C0 = np.broadcast_to(Cb[:, None, None, None], (N, 1, ny, nx)).copy()
    v0 = np.zeros((3, 1, ny, nx))
    v0[0], v0[1] = vb
    st = B.init_state(prm, geo, C0, v0)
    f0, g0, gh0 = st.f.copy(), st.g.copy(), st.ghost.copy()
    st = B.run(prm, geo, st, 20)
    assert np.abs(st.f - f0)[:, geo.fluid].max() < 1e-15
    assert np.abs(st.g - g0)[:, :, geo.fluid].max() < 1e-14
    assert np.abs(st.ghost - gh0).max() < 1e-15


def test_outflow_column_relaxes_towards_the_upstream_value():
    # implicit upwind: the last column moves by U / (1 + U) of its distance to the column
    # upstream per step (a swap of the two weights would move it almost all the way)
    N, nx, ny, u = 2, 10, 4, 0.02
    sig = np.array([[0.0, 0.005], [0.005, 0.0]])
    p = W.base_params(W.D2Q9, nx, ny, 1, N, sig, 1.0)
    prm = lbm.Params(p)
    node = np.zeros((1, ny, nx), int)
    node[..., 0] = B.INLET0
    geo = B.Geometry(prm, node, [[u, 0.0, 1.0, 0.0]], outflow=True)
    C0 = np.zeros((N, 1, ny, nx))
    C0[0] = 1.0
    C0[0, ..., -1], C0[1, ..., -1] = 0.8, 0.2
    v0 = np.zeros((3, 1, ny, nx))
    v0[0] = u
    st = B.step(prm, geo, B.init_state(prm, geo, C0, v0))
    C, _, _, _ = B.fields(prm, geo, st)
    expect = (0.8 + u * 1.0) / (1 + u)
    assert np.abs(C[0, 0, :, -1] - expect).max() < 2e-3
    # the ghost column follows the boundary column by the same small step
    moved = (st.ghost[0, 0] - 0.8) / (C[0, 0, :, -1] - 0.8)
    assert np.abs(moved - u / (1 + u)).max() < 2e-3


def test_outflow_plane_relaxes_towards_the_upstream_value_d3q19():
    # the same implicit upwind rule on the D3Q19 outflow plane and its ghost plane
    N, nx, ny, nz, u = 2, 10, 4, 3, 0.02
    sig = np.array([[0.0, 0.005], [0.005, 0.0]])
    p = W.base_params(W.D3Q19, nx, ny, nz, N, sig, 1.0)
    prm = lbm.Params(p)
    node = np.zeros((nz, ny, nx), int)
    node[..., 0] = B.INLET0
    geo = B.Geometry(prm, node, [[u, 0.0, 0.0, 1.0, 0.0]], outflow=True)
    C0 = np.zeros((N, nz, ny, nx))
    C0[0] = 1.0
    C0[0, ..., -1], C0[1, ..., -1] = 0.8, 0.2
    v0 = np.zeros((3, nz, ny, nx))
    v0[0] = u
    st = B.step(prm, geo, B.init_state(prm, geo, C0, v0))
    C, _, _, _ = B.fields(prm, geo, st)
    expect = (0.8 + u * 1.0) / (1 + u)
    assert np.abs(C[0, :, :, -1] - expect).max() < 2e-3
    moved = (st.ghost[0] - 0.8) / (C[0, :, :, -1] - 0.8)
    assert np.abs(moved - u / (1 + u)).max() < 2e-3


def test_geometry_validation():
    p = W.base_params(W.D2Q9, 8, 4, 1, 2, np.array([[0, 0.005], [0.005, 0]]), 1.0)
    prm = lbm.Params(p)
    node = np.zeros((1, 4, 8), int)
    with pytest.raises(ValueError):
        B.Geometry(prm, node, outflow=True)                 # fluid in column 0
    node[..., 0] = B.SOLID
    node[0, 0, 3] = B.INLET0
    with pytest.raises(ValueError):
        B.Geometry(prm, node)                               # inlet class without a table row
    B.Geometry(prm, node, [[0.0, 0.0, 1.0, 0.0]], outflow=True)


def test_inlet_injects_its_composition_at_the_inflow_rate():
    # reading of the volume-fraction inlet: links from the inlet carry the equilibrium of the
    # prescribed state, so a channel fed at (u, 0) with C_b gains C_b u H of the inlet component
    # per step (H rows) once the first transient has passed; the printed anti-bounce-back would
    # carry in only the interior's own composition (no gain here)
    N, nx, ny, u = 2, 40, 6, 0.02
    sig = np.array([[0.0, 0.005], [0.005, 0.0]])
    prm = lbm.Params(W.base_params(W.D2Q9, nx, ny, 1, N, sig, 0.8))
    node = np.zeros((1, ny, nx), int)
    node[..., 0] = B.INLET0
    rates = []
    for cb in (1.0, 0.4):
        geo = B.Geometry(prm, node, [[u, 0.0, 1.0 - cb, cb]], outflow=True)
        C0 = np.zeros((N, 1, ny, nx))
        C0[0] = 1.0
        v0 = np.zeros((3, 1, ny, nx))
        v0[0] = u
        st = B.run(prm, geo, B.init_state(prm, geo, C0, v0), 100)
        m0 = B.fields(prm, geo, st)[0][1][geo.fluid].sum()
        st = B.run(prm, geo, st, 150)
        m1 = B.fields(prm, geo, st)[0][1][geo.fluid].sum()
        rates.append((m1 - m0) / 150 / (u * ny * cb))
    assert all(0.9 < r < 1.05 for r in rates), rates


def _mixture3d(nx, ny, nz, seed):
    x, y, z = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float), np.arange(nz, dtype=float),
                          indexing="xy")
    x, y, z = (np.transpose(a, (2, 0, 1)) for a in (x, y, z))      # (nz, ny, nx)
    rng = np.random.default_rng(seed)
    c = rng.uniform(2, [nx - 2, ny - 2, nz - 2], size=(2, 3))
    a = W.tanh_step(2.5 - np.sqrt((x - c[0, 0]) ** 2 + (y - c[0, 1]) ** 2 + (z - c[0, 2]) ** 2))
    b = (1 - a) * W.tanh_step(2.0 - np.sqrt((x - c[1, 0]) ** 2 + (y - c[1, 1]) ** 2 + (z - c[1, 2]) ** 2))
    return np.stack([1 - a - b, a, b])


def test_solid_layers_are_the_edge_walls_d3q19():
    # D3Q19: a box bounded by edge walls in y and z (Eqs. 44-45, the gradient rule at the edge)
    # and the same box with solid layers around it in y and z, periodic there
    nx, ny, nz = 6, 5, 4
    C = _mixture3d(nx, ny, nz, 7)
    pa = W.base_params(W.D3Q19, nx, ny, nz, 3, _sigma3(), 0.8, walls=(False, True, True), omega_stab=1 / 90)
    pb = W.base_params(W.D3Q19, nx, ny + 2, nz + 2, 3, _sigma3(), 0.8, omega_stab=1 / 90)
    prm_a, prm_b = lbm.Params(pa), lbm.Params(pb)
    node = np.zeros((nz + 2, ny + 2, nx), int)
    node[0] = node[-1] = B.SOLID
    node[:, 0] = node[:, -1] = B.SOLID
    geo = B.Geometry(prm_b, node)
    Cb = np.zeros((3, nz + 2, ny + 2, nx))
    Cb[:, 1:-1, 1:-1] = C
    Cb[0, node == B.SOLID] = 1.0
    sa = lbm.run(prm_a, lbm.init_state(prm_a, C), 12)
    sb = B.run(prm_b, geo, B.init_state(prm_b, geo, Cb), 12)
    np.testing.assert_allclose(sb.f[:, 1:-1, 1:-1], sa.f, rtol=0, atol=1e-15)
    np.testing.assert_allclose(sb.g[:, :, 1:-1, 1:-1], sa.g, rtol=0, atol=1e-15)


def test_interior_block_conserves_every_component_d3q19():
    nx, ny, nz = 10, 8, 7
    p = W.base_params(W.D3Q19, nx, ny, nz, 3, _sigma3(), 0.7, omega_stab=1 / 90, body_force=(2e-5, 0, 0))
    prm = lbm.Params(p)
    node = np.zeros((nz, ny, nx), int)
    node[2:5, 3:6, 4:7] = B.SOLID
    geo = B.Geometry(prm, node)
    st = B.init_state(prm, geo, _mixture3d(nx, ny, nz, 9))
    C0, _, _, _ = B.fields(prm, geo, st)
    st = B.run(prm, geo, st, 20)
    C1, v, _, _ = B.fields(prm, geo, st)
    m0, m1 = C0[:, geo.fluid].sum(axis=1), C1[:, geo.fluid].sum(axis=1)
    np.testing.assert_allclose(m1, m0, rtol=0, atol=1e-12 * nx * ny * nz)
    assert np.abs(v[:, ~geo.fluid]).max() == 0.0
    np.testing.assert_array_equal(C1[:, ~geo.fluid], C0[:, ~geo.fluid])   # solid nodes keep C
    assert np.abs(v[:, geo.fluid]).max() > 1e-6


def test_uniform_inflow_through_to_the_outflow_is_a_fixed_point_d3q19():
    # D3Q19 version of the pin above: inlet plane at x = 0, convective outflow at x = nx - 1
    N, nx, ny, nz = 3, 10, 5, 4
    p = W.base_params(W.D3Q19, nx, ny, nz, N, _sigma3(), 0.8, omega_stab=1 / 90)
    prm = lbm.Params(p)
    node = np.zeros((nz, ny, nx), int)
    node[..., 0] = B.INLET0
    Cb, vb = np.array([0.2, 0.5, 0.3]), (0.01, 0.003, -0.002)
    geo = B.Geometry(prm, node, [[*vb, *Cb]], outflow=True)
    C0 = np.broadcast_to(Cb[:, None, None, None], (N, nz, ny, nx)).copy()
    v0 = np.zeros((3, nz, ny, nx))
    v0[0], v0[1], v0[2] = vb
    st = B.init_state(prm, geo, C0, v0)
    f0, g0, gh0 = st.f.copy(), st.g.copy(), st.ghost.copy()
    assert gh0.shape == (N - 1, nz, ny)
    st = B.run(prm, geo, st, 15)
    assert np.abs(st.f - f0)[:, geo.fluid].max() < 1e-15
    assert np.abs(st.g - g0)[:, :, geo.fluid].max() < 1e-14
    assert np.abs(st.ghost - gh0).max() < 1e-15


def test_uniform_inflow_is_a_fixed_point_d3q19():
    # D3Q19, periodic in x: a uniform mixture moving at v_b (all three components nonzero) fed by
    # an inlet plane at x = 0 holding the same state stays as it is; the fluid leaving at
    # x = nx - 1 meets the inlet plane through the wrap, so the moving-wall rule acts on both
    # faces of the plane
    N, nx, ny, nz = 3, 8, 5, 4
    p = W.base_params(W.D3Q19, nx, ny, nz, N, _sigma3(), 0.8, omega_stab=1 / 90)
    prm = lbm.Params(p)
    node = np.zeros((nz, ny, nx), int)
    node[..., 0] = B.INLET0
    Cb, vb = np.array([0.2, 0.5, 0.3]), (0.01, 0.003, -0.004)
    geo = B.Geometry(prm, node, [[*vb, *Cb]])
    C0 = np.broadcast_to(Cb[:, None, None, None], (N, nz, ny, nx)).copy()
    v0 = np.zeros((3, nz, ny, nx))
    v0[0], v0[1], v0[2] = vb
    st = B.init_state(prm, geo, C0, v0)
    f0, g0 = st.f.copy(), st.g.copy()
    st = B.run(prm, geo, st, 15)
    assert np.abs(st.f - f0)[:, geo.fluid].max() < 1e-15
    assert np.abs(st.g - g0)[:, :, geo.fluid].max() < 1e-14
    C, v, _, _ = B.fields(prm, geo, st)
    np.testing.assert_allclose(v[:, node == B.INLET0], np.array(vb)[:, None] * np.ones((1, ny * nz)), atol=0)


def test_inlet_feeds_a_closed_box_d3q19():
    # an inlet in one face of a box with solid walls elsewhere: the composition C_b enters; and
    # with v_b = 0 and the box's own composition the inlet face acts as a wall (a state at rest
    # stays at rest)
    N, nx, ny, nz = 3, 8, 6, 5
    p = W.base_params(W.D3Q19, nx, ny, nz, N, _sigma3(), 0.8, omega_stab=1 / 90)
    prm = lbm.Params(p)
    node = np.full((nz, ny, nx), B.SOLID, int)
    node[1:-1, 1:-1, 1:-1] = B.FLUID
    node[2:4, 2:4, 0] = B.INLET0                             # a 2 x 2 inlet in the x = 0 face
    Cb, vb = np.array([0.0, 1.0, 0.0]), (0.01, 0.0, 0.0)
    geo = B.Geometry(prm, node, [[*vb, *Cb]])
    C0 = np.zeros((N, nz, ny, nx))
    C0[0] = 1.0
    st = B.init_state(prm, geo, C0)
    C_a, _, _, _ = B.fields(prm, geo, st)
    st = B.run(prm, geo, st, 30)
    C_b, _, _, _ = B.fields(prm, geo, st)
    fl = geo.fluid
    assert C_b[1][fl].sum() > C_a[1][fl].sum() + 0.01          # component 1 came in
    assert np.isfinite(st.f).all() and np.isfinite(st.g).all()
    Cr = np.array([0.3, 0.3, 0.4])
    geo0 = B.Geometry(prm, node, [[0.0, 0.0, 0.0, *Cr]])
    st = B.init_state(prm, geo0, np.broadcast_to(Cr[:, None, None, None], (N, nz, ny, nx)).copy())
    f0, g0 = st.f.copy(), st.g.copy()
    st = B.run(prm, geo0, st, 10)
    assert np.abs(st.f - f0)[:, fl].max() < 1e-15 and np.abs(st.g - g0)[:, :, fl].max() < 1e-14
