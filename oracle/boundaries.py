"""Open and complex boundaries of Sec. III C, the conditions that the emulsion and PaLS
applications of Sec. V use, on D2Q9 and D3Q19: solid nodes inside the grid, Dirichlet inlets of
velocity and volume fraction, and the convective outflow.

Oracle code (test infrastructure only): imported by tests, the smoke check and the
benchmark's CPU baseline, never by the product path.

Every site has a node class: 0 fluid, 1 solid, 2 + j inlet j with the prescribed state
(v_b, C_b) of row j of the inlet table.  Non-fluid nodes neither collide nor stream: their
f and g stay as they were set.

solid   Halfway bounce-back for f and g (Eqs. 44-45); in every directional difference a
        neighbour inside a solid node takes the value at x (Sec. III C, the rule of Lee and
        Liu cited there).
inlet   Velocity Dirichlet (the moving-wall bounce-back cited in Sec. III C), rho_b = 1:
        f_k(x, t+1) = f*_kbar(x) + 2 w_k rho_b (e_k . v_b) / c_s^2 for the direction k that
        enters the fluid from the inlet node.  The printed rule carries a minus sign, which
        holds when e_k is the direction of the population that left; with e_k the entering
        direction only the plus sign keeps a uniform flow at v_b unchanged.
        Volume fractions: links from an inlet node carry the equilibrium of the prescribed
        state, g_k(x, t+1) = g^eq_k(C_b, v_b, S_b), with S_b the flux potential of the
        uniform state C_b (Eq. 12 without the Laplacian term).  The printed anti-bounce-back,
        -g*_kbar(x) + 2 g^eq_kbar(C_b, v_b), brings no C_b into the domain under the reading
        of Eq. 40 that keeps the C_i share in the rest population (lbm.g_equilibrium): the
        moving populations carry only C_i s_k(v) and the m S_i terms, so the net flux through
        the link is set by C_i(x), not by C_b.  Directional differences see C_b and E_B(C_b) at
        the inlet node, as Sec. III C asks.
outflow Convective condition on the last column (plane) x = nx - 1 (the convective boundary
        equations of Sec. III C): every population there becomes
        (f(N, t) + U f(N-1, t+1)) / (1 + U), U the mean of sum_k e_kx f_k(t+1) over the fluid
        nodes of column nx - 2 (the F/2 term of Eq. 37 is left out: F at t+1 is not known
        yet).  A ghost column N+1 holds the evolved C_i, convected the same way with
        C_i(N, t+1), and serves the directional differences of column N; it starts equal to
        column N and is solid where column N is.  Column 0 must hold no fluid node, column
        nx - 1 no inlet node, and the x axis no edge wall.

Every choice above that the paper leaves open (rho_b, the sign, the composition inlet, U
without F/2, the ghost's start and class) is a reading of Sec. III C, stated where it is made.
"""
from __future__ import annotations

import copy

import numpy as np

from . import lbm

FLUID, SOLID, INLET0 = 0, 1, 2


class Geometry:
    """Node classes (shape of the grid), inlet table rows (v_b with one component per lattice
    dimension, then C_1..C_N) and the outflow flag."""

    def __init__(self, prm, node, inlets=(), outflow=False):
        D = prm.lat.dim
        self.node = np.asarray(node, dtype=np.int64).reshape(prm.shape)
        tab = np.asarray(inlets, dtype=np.float64).reshape(-1, D + prm.N)
        self.inlets = []
        for row in tab:
            vb = np.zeros(3)
            vb[:D] = row[:D]
            Cb = row[D:].copy()
            # S_b: flux potential of the uniform state C_b (no Laplacian term)
            Sb = prm.tables.bulk_flux_potential(Cb.reshape(prm.N, 1, 1, 1))[:, 0, 0, 0]
            self.inlets.append((vb, Cb, Sb))
        self.outflow = bool(outflow)
        if self.node.min() < 0 or self.node.max() >= INLET0 + len(self.inlets):
            raise ValueError("node class out of range")
        if self.outflow:
            if prm.walls[0]:
                raise ValueError("outflow needs a periodic x axis")
            if (self.node[..., 0] == FLUID).any():
                raise ValueError("outflow: column 0 must hold no fluid node")
            if (self.node[..., -1] >= INLET0).any():
                raise ValueError("outflow: column nx - 1 must hold no inlet node")
        self.fluid = self.node == FLUID


class OpenState(lbm.State):
    def __init__(self, f, g, t=0, ghost=None):
        super().__init__(f, g, t)
        self.ghost = ghost        # (N-1, nz, ny): evolved C of the ghost column, or None


def _with_inlet_values(prm, geo, C):
    C = C.copy()
    for j, (_, Cb, _) in enumerate(geo.inlets):
        C[:, geo.node == INLET0 + j] = Cb[:, None]
    return C


def init_state(prm, geo, C0, v0=None, flux_form="literal"):
    """f = f^eq(P = 0, v0), g = g^eq(C0, v0, S(C0)) (lbm.init_state) with C0 := C_b on the
    inlet nodes; the ghost column starts as column nx - 1."""
    C0 = np.asarray(C0, dtype=np.float64).reshape((prm.N,) + prm.shape)
    C0 = _with_inlet_values(prm, geo, C0)
    sp = copy.copy(prm)
    sp.solid = geo.node == SOLID
    st = lbm.init_state(sp, C0, v0, flux_form=flux_form)
    ghost = C0[prm.evolved][..., -1].copy() if geo.outflow else None
    return OpenState(st.f, st.g, 0, ghost)


def _macroscopic(prm, geo, C, f, flux_form):
    """lbm.macroscopic with the solid rule."""
    ext = copy.copy(prm)
    ext.solid = geo.node == SOLID
    return lbm.macroscopic(ext, C, f, flux_form)


def _macroscopic_out(prm, geo, C, f, ghost, flux_form):
    """lbm.macroscopic with the solid rule on the grid extended by the ghost column."""
    N = prm.N
    gh = np.empty((N,) + prm.shape[:-1] + (1,))
    rest = np.zeros(prm.shape[:-1] + (1,))
    for a, c in enumerate(prm.evolved):
        gh[c] = ghost[a][..., None]
        rest = rest + gh[c]
    gh[prm.implicit] = 1.0 - rest
    Cx = np.concatenate([C, gh], axis=-1)
    fx = np.concatenate([f, np.zeros(f.shape[:-1] + (1,))], axis=-1)
    solid = geo.node == SOLID
    ext = copy.copy(prm)
    ext.nx = prm.nx + 1
    ext.shape = prm.shape[:-1] + (prm.nx + 1,)
    ext.solid = np.concatenate([solid, solid[..., -1:]], axis=-1)
    mac = lbm.macroscopic(ext, Cx, fx, flux_form)
    return {k: (v[..., :prm.nx] if isinstance(v, np.ndarray) else v) for k, v in mac.items()}


def macroscopic(prm, geo, C, f, ghost=None, flux_form="literal"):
    """Fields of every fluid node, with the inlet nodes' v and S set to (v_b, S_b)."""
    mac = (_macroscopic_out(prm, geo, C, f, ghost, flux_form) if geo.outflow
           else _macroscopic(prm, geo, C, f, flux_form))
    for j, (vb, _, Sb) in enumerate(geo.inlets):
        sel = geo.node == INLET0 + j
        mac["v"][:, sel] = vb[:, None]
        mac["S"][:, sel] = Sb[:, None]
    return mac


def _shift(a, e):
    return np.roll(a, shift=(int(e[2]), int(e[1]), int(e[0])), axis=(-3, -2, -1))


def _stream(prm, geo, post, old, velocity_rule):
    """new_k(x) = post_k(x - e_k) from a fluid or inlet node; post_kbar(x) from a solid node or
    beyond an edge wall; for f (velocity_rule) the inlet rule above.  Non-fluid x keeps `old`."""
    lat = prm.lat
    new = np.empty_like(post)
    for k in range(lat.Q):
        e = lat.e[k]
        kb = lat.opp[k]
        src = _shift(geo.node, e)
        wall = lbm._outside_plus(prm, kb)
        val = _shift(post[k], e)
        if velocity_rule:
            for j, (vb, _, _) in enumerate(geo.inlets):
                corr = 2.0 * lat.w[k] * float(np.dot(lat.e[k], vb)) / lbm.CS2
                val = np.where(src == INLET0 + j, post[kb] + corr, val)
        val = np.where(wall | (src == SOLID), post[kb], val)
        new[k] = val
    return np.where(geo.fluid, new, old)


def step(prm, geo, st, flux_form="literal"):
    """One time step (lbm.step with the boundaries above).  Returns the new OpenState."""
    lat = prm.lat
    C = _with_inlet_values(prm, geo, lbm.components(prm, st.g))
    mac = macroscopic(prm, geo, C, st.f, st.ghost, flux_form)
    fpost = lbm.collide_f(lat, st.f, mac["P"], mac["v"], mac["F"], mac["omega_p"], mac["omega_m"])
    gpost = np.empty_like(st.g)
    for a, c in enumerate(prm.evolved):
        geq = lbm.g_equilibrium(lat, C[c], mac["v"], mac["S"][c], prm.m)
        gp = st.g[a] - (st.g[a] - geq) / prm.tau_g
        # an inlet node's outgoing populations are the equilibrium of its prescribed state
        gpost[a] = np.where(geo.node >= INLET0, geq, gp)
    f_new = _stream(prm, geo, fpost, st.f, True)
    g_new = np.stack([_stream(prm, geo, gpost[a], st.g[a], False) for a in range(len(prm.evolved))])
    ghost = None
    if geo.outflow:
        nx = prm.nx
        col = geo.fluid[..., nx - 2]
        jx = sum(lat.e[k, 0] * f_new[k][..., nx - 2] for k in range(lat.Q))
        U = float(jx[col].mean()) if col.any() else 0.0
        tgt = geo.fluid[..., nx - 1]
        f_new[..., nx - 1] = np.where(tgt, (st.f[..., nx - 1] + U * f_new[..., nx - 2]) / (1.0 + U),
                                      f_new[..., nx - 1])
        g_new[..., nx - 1] = np.where(tgt, (st.g[..., nx - 1] + U * g_new[..., nx - 2]) / (1.0 + U),
                                      g_new[..., nx - 1])
        CN = g_new[..., nx - 1].sum(axis=1)                   # evolved C of column N, (N-1, nz, ny)
        ghost = (st.ghost + U * CN) / (1.0 + U)
    return OpenState(f_new, g_new, st.t + 1, ghost)


def run(prm, geo, st, nsteps, flux_form="literal"):
    for _ in range(nsteps):
        st = step(prm, geo, st, flux_form)
    return st


def fields(prm, geo, st, flux_form="literal"):
    """(C, v, P, F_s): fluid nodes as lbm.fields; solid nodes v = P = F_s = 0; inlet nodes
    C = C_b, v = v_b, P = F_s = 0."""
    C = _with_inlet_values(prm, geo, lbm.components(prm, st.g))
    mac = macroscopic(prm, geo, C, st.f, st.ghost, flux_form)
    v, P, Fs = mac["v"].copy(), mac["P"].copy(), mac["Fs"].copy()
    nonfluid = ~geo.fluid
    v[:, nonfluid] = 0.0
    P[nonfluid] = 0.0
    Fs[:, nonfluid] = 0.0
    for j, (vb, _, _) in enumerate(geo.inlets):
        v[:, geo.node == INLET0 + j] = vb[:, None]
    return C, v, P, Fs
