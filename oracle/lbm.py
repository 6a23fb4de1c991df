"""Sec. III of the paper: the lattice Boltzmann scheme, written out literally.

Oracle code (test infrastructure only).  Fields have shape (nz, ny, nx)
(nz = 1 for D2Q9); component stacks have a leading axis.  The stepper keeps
all Q populations f_k, f_0 included, and all populations g_{i,k} of the N-1
evolved components with a general tau_g, and takes one time step in the
order below (Sec. III; the paper spreads the order over its subsections):

  1. C_i = sum_k g_{i,k} for the evolved components (Eq. 41);
     C_implicit = 1 - sum of the evolved ones (Sec. II, below Eq. 3).
  2. Isotropic grad and Laplacian of every C_i (Eqs. 35-36), E_B (Eq. 5) and
     grad E_B; a neighbour inside a wall takes the value at x (Sec. III C).
  3. Flux potential S_i = sum_j alpha_ij (mu_j + phi_j + xi_j) (Eq. 12).
  4. Force F = grad E_B + sum_{i != j} kappa_ij lap C_j grad C_i + F_b (Eq. 34).
  5. rho v = sum_k e_k f_k + F/2 (Eq. 37) and P (Eq. 38) with rho = 1;
     viscosity of the component with the largest C (Eq. 42).
  6. TRT collision of f with forcing (Eqs. 23-30); BGK collision of g
     towards g^eq (Eqs. 39-40).
  7. Streaming of both, halfway bounce-back at walls (Eqs. 44-45), periodic
     wrap on the other edges.

Readings: rho_i = 1, so rho = 1 and grad rho = 0 and
the grad-rho terms of Eqs. 30 and 38 vanish; g^eq of Eq. 40 is read as
C_i (delta_k0 + s_k(v)) -/+ (m S_i terms) (see `g_equilibrium`); f^eq_0 is taken as P/c_s^2 (w_0 - 1) + s_0(v)
(f_0 feeds no moment, so this choice changes no other value; `feq0_sign`
switches to the printed sign); argmax ties go to the lowest index.
"""
from __future__ import annotations

import numpy as np

from .thermo import Tables, bulk_energy

CS2 = 1.0 / 3.0


class Lattice:
    """Velocity set e_k and weights w_k."""

    def __init__(self, q):
        if q == 9:
            # Eqs. 20-21 (the paper's D2Q9 ordering)
            ex = [0, 1, -1, 0, 0, 1, -1, 1, -1]
            ey = [0, 0, 0, 1, -1, 1, -1, -1, 1]
            ez = [0] * 9
            w = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
            self.dim = 2
        elif q == 19:
            # Standard D3Q19 set (Sec. III: "straightforward ... standard route")
            vel = [(0, 0, 0)]
            for a in range(3):
                for s in (1, -1):
                    v = [0, 0, 0]
                    v[a] = s
                    vel.append(tuple(v))
            for a, b in ((0, 1), (0, 2), (1, 2)):
                for sa, sb in ((1, 1), (-1, -1), (1, -1), (-1, 1)):
                    v = [0, 0, 0]
                    v[a], v[b] = sa, sb
                    vel.append(tuple(v))
            ex = [v[0] for v in vel]
            ey = [v[1] for v in vel]
            ez = [v[2] for v in vel]
            w = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12
            self.dim = 3
        else:
            raise ValueError("lattice must be 9 (D2Q9) or 19 (D3Q19)")
        self.Q = q
        self.e = np.array([ex, ey, ez], dtype=np.int64).T          # (Q, 3)
        self.w = np.array(w, dtype=np.float64)
        self.opp = np.array([int(np.nonzero((self.e == -self.e[k]).all(axis=1))[0][0])
                             for k in range(q)])


class Params:
    """Run parameters of one simulation (the dict made by `nfe_workloads`)."""

    def __init__(self, p):
        self.lat = Lattice(p["lattice"])
        self.nx, self.ny, self.nz = int(p["nx"]), int(p["ny"]), int(p["nz"])
        self.walls = tuple(bool(w) for w in p["walls"])
        self.N = int(p["N"])
        self.tau = np.asarray(p["tau"], dtype=np.float64)
        self.lambda_trt = float(p["lambda_trt"])
        self.m = float(p["m"])
        self.tau_g = float(p.get("tau_g", 1.0))
        self.body_force = np.asarray(p["body_force"], dtype=np.float64)
        # a body force acting on one component, in proportion to its volume fraction
        # (F += C_c F_c; the PaLS study of Sec. V pushes only the droplet of fluid 2)
        self.component_force = np.asarray(p.get("component_force", (0.0, 0.0, 0.0)), dtype=np.float64)
        self.component_force_index = int(p.get("component_force_index", 0))
        self.implicit = int(p["implicit"])
        self.evolved = [c for c in range(self.N) if c != self.implicit]
        self.tables = Tables(p["sigma"], p["D"], p["omega_stab"])
        self.shape = (self.nz, self.ny, self.nx)


class State:
    def __init__(self, f, g, t=0):
        self.f = f        # (Q, nz, ny, nx)
        self.g = g        # (N-1, Q, nz, ny, nx), evolved components in order
        self.t = t


# ----------------------------------------------------------------------------
# neighbour access with periodic wrap and the wall rules
# ----------------------------------------------------------------------------

def _outside_plus(prm, k):
    """Boolean field: x + e_k lies beyond a wall (only wall axes can be left)."""
    out = np.zeros(prm.shape, dtype=bool)
    e = prm.lat.e[k]
    sizes = (prm.nx, prm.ny, prm.nz)
    for a in range(3):
        if prm.walls[a] and e[a] != 0:
            coord = np.arange(sizes[a])
            bad = (coord + e[a] < 0) | (coord + e[a] >= sizes[a])
            shp = [1, 1, 1]
            shp[2 - a] = sizes[a]
            out = out | bad.reshape(shp)
    return out


def neighbour(prm, psi, k):
    """psi(x + e_k); periodic wrap, and psi(x) where x + e_k is inside a wall (Sec. III C).

    A run with solid nodes (`prm.solid`, boolean field, or absent) applies the same rule
    where x + e_k is a solid node."""
    e = prm.lat.e[k]
    shift = (-int(e[2]), -int(e[1]), -int(e[0]))
    shifted = np.roll(psi, shift=shift, axis=(-3, -2, -1))
    blocked = _outside_plus(prm, k)
    solid = getattr(prm, "solid", None)
    if solid is not None:
        blocked = blocked | np.roll(solid, shift=shift, axis=(-3, -2, -1))
    return np.where(blocked, psi, shifted)


def grad(prm, psi):
    """Isotropic gradient, Eq. 35; returns shape (3,) + psi.shape."""
    lat = prm.lat
    out = np.zeros((3,) + psi.shape)
    for k in range(1, lat.Q):
        d = neighbour(prm, psi, k) - psi
        for a in range(3):
            if lat.e[k, a] != 0:
                out[a] += lat.w[k] * lat.e[k, a] * d
    return out / CS2


def laplacian(prm, psi):
    """Isotropic Laplacian, Eq. 36."""
    lat = prm.lat
    out = np.zeros(psi.shape)
    for k in range(1, lat.Q):
        out += lat.w[k] * (neighbour(prm, psi, k) - psi)
    return 2.0 * out / CS2


def stream(prm, post):
    """Streaming with halfway bounce-back (Eqs. 44-45).

    post has shape (Q, ...).  new_k(x) = post_k(x - e_k) if x - e_k is a fluid
    node, else post_{kbar}(x).
    """
    lat = prm.lat
    new = np.empty_like(post)
    for k in range(lat.Q):
        e = lat.e[k]
        moved = np.roll(post[k], shift=(int(e[2]), int(e[1]), int(e[0])), axis=(-3, -2, -1))
        src_out = _outside_plus(prm, lat.opp[k])
        new[k] = np.where(src_out, post[lat.opp[k]], moved)
    return new


# ----------------------------------------------------------------------------
# macroscopic quantities and equilibria
# ----------------------------------------------------------------------------

def s_k(lat, v):
    """s_k(v) of Eq. 28 for every k; v has shape (3, ...); returns (Q, ...)."""
    vv = np.sum(v * v, axis=0)
    out = np.empty((lat.Q,) + v.shape[1:])
    for k in range(lat.Q):
        ev = sum(lat.e[k, a] * v[a] for a in range(3))
        out[k] = lat.w[k] * (ev / CS2 + ev * ev / (2 * CS2 * CS2) - vv / (2 * CS2))
    return out


def f_equilibrium(lat, P, v, feq0_sign=-1.0):
    """Eq. 27 with rho = 1; f^eq_0 = P/c_s^2 * sign * (1 - w_0) + s_0 (sign -1 by default)."""
    s = s_k(lat, v)
    feq = np.empty_like(s)
    feq[0] = feq0_sign * (P / CS2) * (1.0 - lat.w[0]) + s[0]
    for k in range(1, lat.Q):
        feq[k] = (P / CS2) * lat.w[k] + s[k]
    return feq


def forcing_terms(lat, v, F):
    """F_k of Eq. 30 with grad rho = 0; returns (Q, ...)."""
    vF = np.sum(v * F, axis=0)
    out = np.empty((lat.Q,) + v.shape[1:])
    for k in range(lat.Q):
        ev = sum(lat.e[k, a] * v[a] for a in range(3))
        eF = sum(lat.e[k, a] * F[a] for a in range(3))
        out[k] = lat.w[k] * (eF / CS2 + (ev * eF - CS2 * vF) / (CS2 * CS2))
    return out


def g_equilibrium(lat, Ci, v, Si, m):
    """Eq. 40 for one component: C_i (delta_k0 + s_k(v)) + (1 - w_0) m S_i (k = 0), - w_k m S_i (k != 0).

    The printed w_k C_i (1 + s_k(v)) is garbled (s_k of Eq. 28 already carries
    w_k).  The reading taken puts the C_i part of the zeroth moment in the rest
    population, as in the cited Zheng et al. (2015) scheme.  Its moments are
    then C_i (Eq. 41), C_i v (the advection of Eq. 3) and, at second order,
    C_i v v - c_s^2 m S_i I, so the Chapman-Enskog limit is Eq. 3 with the flux
    of Eq. 12 and the mobility of Eq. 43.  Spreading w_k C_i over all
    directions instead would add a diffusion c_s^2 (tau_g - 1/2) lap C_i that
    is not in Eq. 3 and dissolves every interface.
    """
    s = s_k(lat, v)
    geq = np.empty((lat.Q,) + Ci.shape)
    for k in range(lat.Q):
        geq[k] = Ci * s[k]
        if k == 0:
            geq[k] += Ci + (1.0 - lat.w[0]) * m * Si
        else:
            geq[k] -= lat.w[k] * m * Si
    return geq


def components(prm, g):
    """All N volume fractions from the evolved populations (Eq. 41 and sum C = 1)."""
    C = np.empty((prm.N,) + prm.shape)
    rest = np.zeros(prm.shape)
    for a, c in enumerate(prm.evolved):
        C[c] = g[a].sum(axis=0)
        rest = rest + C[c]
    C[prm.implicit] = 1.0 - rest
    return C


def macroscopic(prm, C, f, flux_form="literal", force_form="conservative", with_phi=True):
    """Steps 2-5 of the time step at fixed C and f.

    Returns a dict with grad/lap of every component, E_B, grad E_B, S (the
    flux potential of every component), F_s, F, v, P and the omega+/omega-
    fields.
    """
    T = prm.tables
    lat = prm.lat
    N = prm.N
    gradC = np.stack([grad(prm, C[i]) for i in range(N)])        # (N, 3, ...)
    lapC = np.stack([laplacian(prm, C[i]) for i in range(N)])     # (N, ...)
    EB = None
    if flux_form == "literal":
        S = T.flux_potential(C, lapC, with_phi=with_phi)
    elif flux_form == "factored":
        S = T.flux_potential_factored(C, lapC)
    else:
        raise ValueError(flux_form)
    if force_form == "conservative":
        EB = bulk_energy(C, T.beta)
        gEB = grad(prm, EB)
        Fs = gEB.copy()
        for i in range(N):
            for j in range(N):
                if i != j:
                    Fs += T.kappa[i, j] * lapC[j] * gradC[i]
    elif force_form == "nonconservative":
        mu = T.mu(C, lapC)
        Fs = np.zeros((3,) + prm.shape)
        for i in range(N):
            Fs += mu[i] * gradC[i]
        gEB = None
    else:
        raise ValueError(force_form)
    F = Fs + prm.body_force.reshape(3, 1, 1, 1)
    if np.any(prm.component_force != 0.0):
        F = F + prm.component_force.reshape(3, 1, 1, 1) * C[prm.component_force_index]
    j = np.zeros((3,) + prm.shape)
    for k in range(1, lat.Q):
        for a in range(3):
            if lat.e[k, a] != 0:
                j[a] += lat.e[k, a] * f[k]
    v = j + 0.5 * F
    s0 = s_k(lat, v)[0]
    P = CS2 / (1.0 - lat.w[0]) * (f[1:].sum(axis=0) + s0)
    # viscosity of the component with the largest volume fraction (Eq. 42);
    # np.argmax returns the lowest index on ties
    idx = np.argmax(C, axis=0)
    tau_p = prm.tau[idx]
    omega_p = 1.0 / tau_p
    if prm.lambda_trt < 0.0:
        omega_m = omega_p
    else:
        omega_m = 1.0 / (prm.lambda_trt / (tau_p - 0.5) + 0.5)       # Eq. 26
    return dict(gradC=gradC, lapC=lapC, EB=EB, gradEB=gEB, S=S, Fs=Fs, F=F, v=v, P=P,
                omega_p=omega_p, omega_m=omega_m, argmax=idx)


def collide_f(lat, f, P, v, F, omega_p, omega_m, feq0_sign=-1.0):
    """TRT collision with the TRT forcing split (Eqs. 23, 24, 29)."""
    feq = f_equilibrium(lat, P, v, feq0_sign)
    Fk = forcing_terms(lat, v, F)
    post = np.empty_like(f)
    for k in range(lat.Q):
        kb = lat.opp[k]
        fp, fm = 0.5 * (f[k] + f[kb]), 0.5 * (f[k] - f[kb])
        ep, em = 0.5 * (feq[k] + feq[kb]), 0.5 * (feq[k] - feq[kb])
        post[k] = (f[k] - omega_p * (fp - ep) - omega_m * (fm - em)
                   + 0.5 * (1.0 - 0.5 * omega_p) * (Fk[k] + Fk[kb])
                   + 0.5 * (1.0 - 0.5 * omega_m) * (Fk[k] - Fk[kb]))
    return post


# ----------------------------------------------------------------------------
# public entry points
# ----------------------------------------------------------------------------

def round_to_storage(x, fmt):
    """x (float64) rounded to a 16-bit storage format and read back as float64.

    fmt "fp16": IEEE binary16, round to nearest even (numpy's conversion);
    fmt "bf16": the upper half of the binary32 word, x first rounded to binary32 and then its
    16 low bits dropped with round to nearest even (the format keeps 8 significand bits).
    Finite inputs only."""
    x = np.asarray(x, dtype=np.float64)
    if fmt == "fp16":
        return x.astype(np.float16).astype(np.float64)
    if fmt == "bf16":
        u = x.astype(np.float32).view(np.uint32).astype(np.uint64)
        odd = (u >> np.uint64(16)) & np.uint64(1)
        u = (u + np.uint64(0x7FFF) + odd) & np.uint64(0xFFFF0000)
        return u.astype(np.uint32).view(np.float32).astype(np.float64)
    raise ValueError(fmt)


def store_populations(lat, f, fmt, scale_exp=0):
    """f as a library keeps it between steps when f is stored in 16 bits (a reading of the
    paper, which stores f in full precision: f_k of this pressure-based scheme vanish at rest,
    so f_k / w_k is stored, times 2^scale_exp for FP16): every f_k with k != 0 is replaced by
    round(f_k / w_k 2^s) w_k 2^-s.  f_0 is untouched (it enters no moment and is not stored).
    fmt None returns f unchanged."""
    if fmt is None:
        return f
    out = f.copy()
    sc = 2.0 ** scale_exp if fmt == "fp16" else 1.0
    for k in range(1, lat.Q):
        out[k] = round_to_storage(f[k] / lat.w[k] * sc, fmt) * lat.w[k] / sc
    return out


def init_state(prm, C0, v0=None, flux_form="literal", f_storage=None, scale_exp=0):
    """f = f^eq(P = 0, v0) and g = g^eq(C0, v0, S(C0)) at t = 0 (f in the storage format
    f_storage, see `store_populations`)."""
    lat = prm.lat
    C0 = np.asarray(C0, dtype=np.float64).reshape((prm.N,) + prm.shape)
    C = C0.copy()
    rest = np.zeros(prm.shape)
    for c in prm.evolved:
        rest = rest + C[c]
    C[prm.implicit] = 1.0 - rest
    v = np.zeros((3,) + prm.shape) if v0 is None else np.asarray(v0, dtype=np.float64).reshape((3,) + prm.shape)
    f = f_equilibrium(lat, np.zeros(prm.shape), v)
    lapC = np.stack([laplacian(prm, C[i]) for i in range(prm.N)])
    if flux_form == "factored":
        S = prm.tables.flux_potential_factored(C, lapC)
    else:
        S = prm.tables.flux_potential(C, lapC)
    g = np.stack([g_equilibrium(lat, C[c], v, S[c], prm.m) for c in prm.evolved])
    return State(store_populations(lat, f, f_storage, scale_exp), g, 0)


def step(prm, st, flux_form="literal", force_form="conservative", with_phi=True, feq0_sign=-1.0,
         f_storage=None, scale_exp=0):
    """Advance one time step (steps 1-7 above).  Returns the new State; with f_storage the
    streamed f is kept in that 16-bit format (`store_populations`)."""
    lat = prm.lat
    C = components(prm, st.g)
    mac = macroscopic(prm, C, st.f, flux_form, force_form, with_phi)
    fpost = collide_f(lat, st.f, mac["P"], mac["v"], mac["F"], mac["omega_p"], mac["omega_m"], feq0_sign)
    gpost = np.empty_like(st.g)
    for a, c in enumerate(prm.evolved):
        geq = g_equilibrium(lat, C[c], mac["v"], mac["S"][c], prm.m)
        gpost[a] = st.g[a] - (st.g[a] - geq) / prm.tau_g
    f_new = store_populations(lat, stream(prm, fpost), f_storage, scale_exp)
    g_new = np.stack([stream(prm, gpost[a]) for a in range(len(prm.evolved))])
    return State(f_new, g_new, st.t + 1)


def run(prm, st, nsteps, **kw):
    for _ in range(nsteps):
        st = step(prm, st, **kw)
    return st


def fields(prm, st, flux_form="literal", force_form="conservative"):
    """(C, v, P) at the current state: C of all N components, v (3, ...), P."""
    C = components(prm, st.g)
    mac = macroscopic(prm, C, st.f, flux_form, force_form)
    return C, mac["v"], mac["P"], mac


def diagnostics(prm, st, flux_form="literal", force_form="conservative"):
    """Global sums in float64: mass per component, momentum sum v, sum F_s, sum |F_s|."""
    C, v, P, mac = fields(prm, st, flux_form, force_form)
    speed = np.sqrt(np.sum(v * v, axis=0))
    return dict(
        step=st.t,
        mass=C.reshape(prm.N, -1).sum(axis=1),
        momentum=v.reshape(3, -1).sum(axis=1),
        force_sum=mac["Fs"].reshape(3, -1).sum(axis=1),
        force_abs_sum=np.abs(mac["Fs"]).reshape(3, -1).sum(axis=1),
        max_abs_C=np.abs(C).reshape(prm.N, -1).max(axis=1),
        min_C=C.reshape(prm.N, -1).min(axis=1),
        max_speed=float(speed.max()),
        nonfinite=int(not (np.isfinite(st.f).all() and np.isfinite(st.g).all())),
    )
