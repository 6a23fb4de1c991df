"""Seeded synthetic inputs for the N-component free-energy LBM.

This module is the one piece shared by the oracle, the tests and the
benchmark.  It holds no arithmetic of the method itself: it only builds
initial volume-fraction fields (tanh-smoothed discs, layers and half-spaces,
or seeded random mixtures), surface-tension matrices and run parameters, in
FP64 on the host, with numpy's PCG64 generator.  Neither the oracle nor the
CUDA library draws random numbers, so both sides always see identical inputs.

Array convention: every field has shape (nz, ny, nx) (nz = 1 for 2-D), so a
C-order ravel gives the x-fastest site index used by the C ABI.  A field
stack for N components has shape (N, nz, ny, nx).

Interface profile: a "tanh interface of width 2 lu" is read as
C = 1/2 (1 + tanh(d / 2)) with d the signed distance, which is the D = 4
equilibrium profile 1/2 (1 + tanh(2 d / D)) of the free energy in Sec. II.
Interfaces are placed half-way between nodes so that no node starts with two
equal largest volume fractions (the viscosity rule of Sec. III B picks the
largest one).
"""
from __future__ import annotations

import numpy as np

D2Q9 = 9
D3Q19 = 19

__all__ = [
    "D2Q9", "D3Q19", "tanh_step", "base_params", "lens_2d", "spinodal_2d",
    "layered_poiseuille", "janus_3d", "janus_2d", "droplet_2d", "planar_2d",
    "batch_sweep", "random_sigma", "random_simplex_points", "phase_separation_2d", "CONFIGS",
    "open_channel_2d", "emulsion_2d", "porous_channel_2d", "porous_3d", "inlet_channel_3d", "pals_2d", "FLUID", "SOLID", "INLET0",
]

# node classes of a geometry (one byte per site)
FLUID, SOLID, INLET0 = 0, 1, 2


def tanh_step(d):
    """1/2 (1 + tanh(d/2)): 1 deep on the positive side of a width-2 interface."""
    return 0.5 * (1.0 + np.tanh(0.5 * np.asarray(d, dtype=np.float64)))


def _coords(nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64),
                          np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def random_sigma(rng, N, lo=0.004, hi=0.012):
    """Symmetric N x N surface-tension matrix, off-diagonal U(lo, hi), zero diagonal."""
    s = np.zeros((N, N))
    for i in range(N):
        for j in range(i + 1, N):
            s[i, j] = s[j, i] = rng.uniform(lo, hi)
    return s


def random_simplex_points(rng, N, count, absent=None):
    """Random points on the unit simplex sum_i C_i = 1 (component `absent` set to 0)."""
    x = rng.uniform(0.0, 1.0, size=(count, N))
    if absent is not None:
        x[:, absent] = 0.0
    return x / x.sum(axis=1, keepdims=True)


def base_params(lattice, nx, ny, nz, N, sigma, tau, *, walls=(False, False, False),
                lambda_trt=-1.0, m=1.0 / 50.0, D=4.0, omega_stab=float("nan"),
                body_force=(0.0, 0.0, 0.0), implicit=None, name=""):
    sigma = np.asarray(sigma, dtype=np.float64)
    tau = np.asarray(tau, dtype=np.float64)
    if tau.ndim == 0:
        tau = np.full(N, float(tau))
    return dict(name=name, lattice=lattice, nx=nx, ny=ny, nz=nz,
                walls=tuple(bool(w) for w in walls), N=N, sigma=sigma, tau=tau,
                lambda_trt=float(lambda_trt), m=float(m), D=float(D),
                omega_stab=float(omega_stab),
                body_force=tuple(float(b) for b in body_force),
                implicit=(N - 1 if implicit is None else int(implicit)))


def lens_2d(nx=64, ny=64, radius=12.0, sigma3=(0.01, 0.008, 0.008), tau=1.0, m=0.05,
            extra_sigma=None, N=3, walls_y=True):
    """Liquid lens: C1 below, C2 above a horizontal interface, a disc of C3 on it.

    Defaults are the 64 x 64 lens (periodic in x, walls in y) with
    (sigma12, sigma13, sigma23) = (0.01, 0.008, 0.008), tau = 1, m = 0.05.
    For N > 3 the extra components are small discs of radius ny/8 placed in
    the lower fluid, each with its own sigma row from `extra_sigma`.
    """
    x, y, z = _coords(nx, ny, 1)
    yc = ny / 2.0 - 0.5
    xc = nx / 2.0 - 0.5
    lower = tanh_step(yc - y)
    disc = tanh_step(radius - np.hypot(x - xc, y - yc))
    C = np.zeros((N, 1, ny, nx))
    C[2] = disc
    C[0] = lower * (1.0 - disc)
    C[1] = (1.0 - lower) * (1.0 - disc)
    s12, s13, s23 = sigma3
    sigma = np.zeros((N, N))
    sigma[0, 1] = sigma[1, 0] = s12
    sigma[0, 2] = sigma[2, 0] = s13
    sigma[1, 2] = sigma[2, 1] = s23
    if N > 3:
        r = ny / 8.0
        for e in range(3, N):
            cx = (e - 2) * nx / (N - 1) - 0.5
            cy = ny / 4.0 - 0.5
            d = tanh_step(r - np.hypot(x - cx, y - cy))
            C[:3] *= (1.0 - d)
            C[e] = d
            for j in range(N):
                if j != e:
                    val = extra_sigma[e][j] if extra_sigma is not None else 0.005
                    sigma[e, j] = sigma[j, e] = val
    p = base_params(D2Q9, nx, ny, 1, N, sigma, tau, walls=(False, walls_y, False), m=m,
                    name=f"lens_{nx}x{ny}_N{N}")
    p["C0"] = C
    return p


def spinodal_2d(nx=512, ny=512, N=4, seed=1002, amp=0.02, sigma=0.005, tau=0.8, m=0.1):
    """Quaternary spinodal mixture: C_i = 1/N + U(-amp, amp), renormalised to sum 1."""
    rng = np.random.default_rng(seed)
    C = 1.0 / N + rng.uniform(-amp, amp, size=(N, 1, ny, nx))
    C /= C.sum(axis=0, keepdims=True)
    sig = np.full((N, N), float(sigma))
    np.fill_diagonal(sig, 0.0)
    p = base_params(D2Q9, nx, ny, 1, N, sig, tau, m=m, name=f"spinodal_{nx}x{ny}_N{N}")
    p["C0"] = C
    return p


def phase_separation_2d(nx=400, ny=400, N=4, seed=1013, sigma=0.005, tau=1.0, m=0.1):
    """Phase-separation start of Sec. IV: C_i ~ U(0, 2/N) on every site, renormalised to sum 1;
    all sigma_ij equal, eta_i = 1/6 (tau = 1)."""
    rng = np.random.default_rng(seed)
    C = rng.uniform(0.0, 2.0 / N, size=(N, 1, ny, nx))
    C /= C.sum(axis=0, keepdims=True)
    sig = np.full((N, N), float(sigma))
    np.fill_diagonal(sig, 0.0)
    p = base_params(D2Q9, nx, ny, 1, N, sig, tau, m=m, name=f"phase_separation_{nx}x{ny}_N{N}")
    p["C0"] = C
    return p


def layered_poiseuille(nx=32, ny=32, nz=192, taus=(0.6, 0.7, 0.8, 0.9, 1.0, 1.2),
                       force=1e-6, lattice=D3Q19, absent=True, sigma=0.005, m=1.0 / 50.0):
    """Equal fluid layers stacked along the wall-normal axis with a body force along x.

    3-D (D3Q19): walls at the z ends, layers along z.  2-D (D2Q9, nz must be 1):
    walls at the y ends, layers along y.  With `absent`, one more component is
    added that is identically zero; it is an evolved component and layer 0 is
    the implicit one (C_implicit = 1 - sum of the others).
    """
    L = len(taus)
    if lattice == D3Q19:
        x, y, z = _coords(nx, ny, nz)
        s, W = z, nz
        walls = (False, False, True)
    else:
        assert nz == 1
        x, y, z = _coords(nx, ny, 1)
        s, W = y, ny
        walls = (False, True, False)
    N = L + (1 if absent else 0)
    width = W / L
    C = np.zeros((N,) + s.shape)
    H = [tanh_step(s - (b * width - 0.5)) for b in range(1, L)]
    C[0] = 1.0 - H[0]
    for lay in range(1, L - 1):
        C[lay] = H[lay - 1] - H[lay]
    C[L - 1] = H[L - 2]
    tau = list(taus) + ([1.0] if absent else [])
    sig = np.full((N, N), float(sigma))
    np.fill_diagonal(sig, 0.0)
    p = base_params(lattice, nx, ny, nz if lattice == D3Q19 else 1, N, sig, tau,
                    walls=walls, lambda_trt=3.0 / 16.0, m=m,
                    body_force=(force, 0.0, 0.0), implicit=0,
                    name=f"poiseuille_{nx}x{ny}x{nz}_N{N}")
    p["C0"] = C
    p["layer_width"] = width
    return p


def _janus_fields(x, y, z, centres, pairs, radius, N, split_axis=0):
    C = np.zeros((N,) + x.shape)
    for (cx, cy, cz), (a, b) in zip(centres, pairs):
        r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2)
        drop = tanh_step(radius - r)
        coord = (x, y, z)[split_axis] - (cx, cy, cz)[split_axis]
        h = tanh_step(coord)
        C[a] += drop * (1.0 - h)
        C[b] += drop * h
    C[0] = 1.0 - C[1:].sum(axis=0)
    return C


def janus_3d(n=256, radius=None, seed=1004, N=4, tau=1.0, m=1.0 / 50.0):
    """Four Janus droplets (two components each, split by the plane x = x_c) in matrix C1.

    radius in lattice units; the default n / 8 is the 256^3 layout's radius 32 at any size.
    """
    if radius is None:
        radius = n / 8.0
    rng = np.random.default_rng(seed)
    sig = random_sigma(rng, N)
    x, y, z = _coords(n, n, n)
    q = n / 4.0
    centres = [(q - 0.5, q - 0.5, q - 0.5), (3 * q - 0.5, 3 * q - 0.5, q - 0.5),
               (q - 0.5, 3 * q - 0.5, 3 * q - 0.5), (3 * q - 0.5, q - 0.5, 3 * q - 0.5)]
    pairs = [(1, 2), (2, 3), (1, 3), (1, 2)]
    C = _janus_fields(x, y, z, centres, pairs, radius, N)
    p = base_params(D3Q19, n, n, n, N, sig, tau, m=m, name=f"janus3d_{n}^3_N{N}")
    p["C0"] = C
    p["centres"] = centres
    p["radius"] = radius
    return p


def janus_2d(nx=100, ny=100, radius=20.0, offset=25.0, tau=1.0, m=1.0 / 50.0, sigma=None):
    """Janus droplet of Sec. IV A: fluid 2 disc in the centre, discs of 3 and 4 at +/- offset.

    Overlaps are removed in the order 2, 3, 4 (later discs take only what is
    left).  Default tensions: sigma14 = sigma24 = 0.0095, the rest 0.005.
    """
    x, y, z = _coords(nx, ny, 1)
    xc, yc = nx / 2.0 - 0.5, ny / 2.0 - 0.5
    d2 = tanh_step(radius - np.hypot(x - xc, y - yc))
    d3 = tanh_step(radius - np.hypot(x - xc - offset, y - yc)) * (1.0 - d2)
    d4 = tanh_step(radius - np.hypot(x - xc + offset, y - yc)) * (1.0 - d2 - d3)
    C = np.zeros((4, 1, ny, nx))
    C[1], C[2], C[3] = d2, d3, d4
    C[0] = 1.0 - C[1:].sum(axis=0)
    if sigma is None:
        sigma = np.full((4, 4), 0.005)
        sigma[0, 3] = sigma[3, 0] = 0.0095
        sigma[1, 3] = sigma[3, 1] = 0.0095
        np.fill_diagonal(sigma, 0.0)
    p = base_params(D2Q9, nx, ny, 1, 4, sigma, tau, m=m, name=f"janus2d_{nx}x{ny}")
    p["C0"] = C
    return p


def droplet_2d(n=128, radius=20.0, sigma=0.005, tau=1.0, m=1.0 / 50.0):
    """Binary droplet (component 1) of the given radius in component 0, periodic box."""
    x, y, z = _coords(n, n, 1)
    c = n / 2.0 - 0.5
    d = tanh_step(radius - np.hypot(x - c, y - c))
    C = np.stack([1.0 - d, d])
    sig = np.array([[0.0, sigma], [sigma, 0.0]])
    p = base_params(D2Q9, n, n, 1, 2, sig, tau, m=m, name=f"droplet_{n}_R{radius}")
    p["C0"] = C
    p["radius"] = radius
    p["centre"] = (c, c)
    return p


def planar_2d(nx=4, ny=64, sigma=0.005, tau=1.0, m=1.0 / 50.0, offset=0.0, width=2.0):
    """Binary slab: component 1 for |y - yc| < ny/4, with tanh edges of width `width` lu."""
    x, y, z = _coords(nx, ny, 1)
    yc = ny / 2.0 - 0.5
    a = 0.5 * (1.0 + np.tanh((ny / 4.0 - np.abs(y - yc) + offset) / width))
    C = np.stack([1.0 - a, a])
    sig = np.array([[0.0, sigma], [sigma, 0.0]])
    p = base_params(D2Q9, nx, ny, 1, 2, sig, tau, m=m, name=f"planar_{nx}x{ny}")
    p["C0"] = C
    return p


def open_channel_2d(nx=70, ny=36, N=3, seed=1021, tau=0.8, m=1.0 / 50.0, outflow=True):
    """Small open channel with every boundary kind: solid rows at y = 0 and y = ny - 1, a solid
    post in the middle, two inlets on the left edge (column 0, the rest of it solid) with
    different compositions and velocities, one inlet in the top wall, and (optionally) the
    convective outflow on the right edge.  The interior starts as a seeded smooth mixture."""
    rng = np.random.default_rng(seed)
    sig = random_sigma(rng, N)
    node = np.zeros((1, ny, nx), dtype=np.uint8)
    node[:, 0, :] = SOLID
    node[:, -1, :] = SOLID
    node[:, :, 0] = SOLID
    if not outflow:
        node[:, :, -1] = SOLID
    h = (ny - 2) // 2
    node[:, 1:1 + h, 0] = INLET0                 # inlet 0: lower half of the left edge
    node[:, 1 + h:ny - 1, 0] = INLET0 + 1        # inlet 1: upper half
    a0 = nx // 3
    node[:, -1, a0:a0 + 6] = INLET0 + 2          # inlet 2: in the top wall, flowing down
    px, py = nx // 2, ny // 2
    node[:, py - 3:py + 2, px - 2:px + 1] = SOLID
    pts = random_simplex_points(rng, N, 3)
    inlets = np.zeros((3, 2 + N))
    inlets[0, :2], inlets[1, :2], inlets[2, :2] = (0.01, 0.0), (0.006, 0.002), (0.0, -0.008)
    inlets[:, 2:] = pts
    x, y, z = _coords(nx, ny, 1)
    C = np.empty((N, 1, ny, nx))
    for i in range(N):
        kx, ky, ph = rng.uniform(1, 3), rng.uniform(1, 3), rng.uniform(0, 2 * np.pi)
        C[i] = 1.0 + 0.6 * np.sin(2 * np.pi * kx * x / nx + ph) * np.cos(2 * np.pi * ky * y / ny)
    C /= C.sum(axis=0, keepdims=True)
    p = base_params(D2Q9, nx, ny, 1, N, sig, tau, m=m, omega_stab=1.0 / 90.0, name=f"open_channel_{nx}x{ny}_N{N}")
    p["C0"] = C
    p["geometry"] = dict(node=node, inlets=inlets, outflow=bool(outflow))
    return p


def porous_channel_2d(nx=4096, ny=1024, N=4, seed=1031, pitch=16, post=4, u=0.01, tau=0.8, m=0.1):
    """A large channel through a square lattice of solid posts (post x post sites every pitch
    sites), solid rows at y = 0 and ny - 1, an inlet column at x = 0 feeding component 0 at
    (u, 0), and the convective outflow at x = nx - 1; the interior starts as the seeded
    spinodal mixture (C_i = 1/N + U(-0.02, 0.02), renormalised).  A throughput case for the
    geometry form of the step at a size far beyond L2."""
    rng = np.random.default_rng(seed)
    node = np.zeros((1, ny, nx), dtype=np.uint8)
    y, x = np.mgrid[0:ny, 0:nx]
    node[0][((x % pitch) >= pitch // 2) & ((x % pitch) < pitch // 2 + post)
            & ((y % pitch) >= pitch // 2) & ((y % pitch) < pitch // 2 + post)] = SOLID
    node[:, 0, :] = SOLID
    node[:, -1, :] = SOLID
    node[:, :, 0] = SOLID
    node[:, 1:-1, 0] = INLET0
    inlets = np.zeros((1, 2 + N))
    inlets[0, 0] = u
    inlets[0, 2] = 1.0
    C = 1.0 / N + rng.uniform(-0.02, 0.02, size=(N, 1, ny, nx))
    C /= C.sum(axis=0, keepdims=True)
    sig = np.full((N, N), 0.005)
    np.fill_diagonal(sig, 0.0)
    p = base_params(D2Q9, nx, ny, 1, N, sig, tau, m=m, name=f"porous_{nx}x{ny}_N{N}")
    p["C0"] = C
    p["geometry"] = dict(node=node, inlets=inlets, outflow=True)
    return p


def porous_3d(nx=40, ny=30, nz=20, N=4, seed=1041, walls=(False, False, True), tau=0.8, m=1.0 / 50.0,
              pitch=10, post=3, body_force=(1e-6, 0.0, 0.0)):
    """A D3Q19 porous block: solid cubes of post^3 sites every pitch sites (one per pitch^3 cell)
    plus one solid slab across the grid at x in [nx/2, nx/2 + 2) with a square window of side
    ny/3 in its middle; the given edge walls; a seeded smooth mixture of N components (two
    tanh spheres in a matrix) driven by a small body force along x.  Fluid and solid nodes only."""
    rng = np.random.default_rng(seed)
    sig = random_sigma(rng, N)
    # broadcast coordinates (nz, ny, nx)
    z, y, x = (a.astype(np.float64) for a in np.ogrid[0:nz, 0:ny, 0:nx])
    node = np.zeros((nz, ny, nx), dtype=np.uint8)
    o = pitch // 2
    node[((x % pitch) >= o) & ((x % pitch) < o + post) & ((y % pitch) >= o) & ((y % pitch) < o + post)
         & ((z % pitch) >= o) & ((z % pitch) < o + post)] = SOLID
    w = max(ny // 3, 2)
    slab = (x >= nx // 2) & (x < nx // 2 + 2)
    window = (np.abs(y - (ny - 1) / 2.0) < w / 2.0) & (np.abs(z - (nz - 1) / 2.0) < w / 2.0)
    node[slab & ~window] = SOLID
    C = np.zeros((N, nz, ny, nx))
    centres = rng.uniform(0.2, 0.8, size=(2, 3)) * np.array([nx, ny, nz])
    radius = min(nx, ny, nz) / 5.0
    rest = np.ones((nz, ny, nx))
    for i, c in enumerate(centres):
        d = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
        ci = rest * tanh_step(radius - d)
        C[1 + i % (N - 1)] += ci
        rest -= ci
    C[0] = rest
    np.clip(C, 0.0, None, out=C)
    C /= C.sum(axis=0, keepdims=True)
    p = base_params(D3Q19, nx, ny, nz, N, sig, tau, walls=walls, m=m, omega_stab=1.0 / 90.0,
                    body_force=body_force, name=f"porous3d_{nx}x{ny}x{nz}_N{N}")
    p["C0"] = C
    p["geometry"] = dict(node=node, inlets=np.zeros((0, 2 + N)), outflow=False)
    return p


def inlet_channel_3d(nx=40, ny=18, nz=14, N=3, seed=1051, tau=0.8, m=1.0 / 50.0, outflow=False):
    """A D3Q19 channel, periodic in x, with solid planes at y = 0, ny - 1 and z = 0, nz - 1, a
    solid post in the middle, and the plane x = 0 split into two inlets (lower and upper half in
    y) of different compositions and velocities (every velocity component nonzero), plus a third
    inlet patch in the upper y plane; the interior starts as a seeded smooth mixture.  Without the
    outflow the fluid leaving at x = nx - 1 meets the inlet plane through the wrap; with it the
    plane x = nx - 1 takes the convective outflow."""
    rng = np.random.default_rng(seed)
    sig = random_sigma(rng, N)
    node = np.zeros((nz, ny, nx), dtype=np.uint8)
    node[0] = node[-1] = SOLID
    node[:, 0] = node[:, -1] = SOLID
    h = ny // 2
    node[1:-1, 1:h, 0] = INLET0
    node[1:-1, h:-1, 0] = INLET0 + 1
    node[nz // 2 - 2:nz // 2 + 2, -1, nx // 3:nx // 3 + 5] = INLET0 + 2
    node[nz // 2 - 2:nz // 2 + 1, ny // 2 - 2:ny // 2 + 2, nx // 2 - 1:nx // 2 + 2] = SOLID
    pts = random_simplex_points(rng, N, 3)
    inlets = np.zeros((3, 3 + N))
    inlets[0, :3], inlets[1, :3], inlets[2, :3] = (0.01, 0.002, -0.001), (0.006, -0.002, 0.003), (0.001, -0.008, 0.0)
    inlets[:, 3:] = pts
    x, y, z = _coords(nx, ny, nz)
    C = np.empty((N, nz, ny, nx))
    for i in range(N):
        kx, ky, kz, ph = rng.uniform(1, 3), rng.uniform(1, 3), rng.uniform(1, 2), rng.uniform(0, 2 * np.pi)
        C[i] = 1.0 + 0.6 * np.sin(2 * np.pi * kx * x / nx + ph) * np.cos(2 * np.pi * ky * y / ny) * np.cos(2 * np.pi * kz * z / nz)
    C /= C.sum(axis=0, keepdims=True)
    p = base_params(D3Q19, nx, ny, nz, N, sig, tau, m=m, omega_stab=1.0 / 90.0, name=f"inlet_channel3d_{nx}x{ny}x{nz}_N{N}")
    p["C0"] = C
    p["geometry"] = dict(node=node, inlets=inlets, outflow=bool(outflow))
    return p


def pals_2d(nx=400, ny=140, force=3e-7, m=1.0 / 50.0):
    """The patterned liquid surface of Sec. V, N = 4 (fluids 1..4 = components 0..3): halfway
    walls at the bottom and top (y), periodic in x; eight stripes of alternating lubricants 3 and
    4 of height 15 on the bottom wall; solid posts of 2 x 5 sites on the wall at each
    lubricant-lubricant interface; a hemispherical droplet of fluid 2 of radius 60 resting on
    the lubricant, in fluid 1; a horizontal body force acting on fluid 2 only (F = C_2 F_b).
    sigma_13 = sigma_14 = sigma_23 = sigma_24 = 0.01, sigma_12 = sigma_34 = 0.005, Omega = 1/90,
    eta = (2/300, 0.1, 2/3, 2/3) (tau = 3 eta + 1/2), Lambda_TRT = 3/16.  Interfaces are tanh
    profiles of width 2 lu; the stripe and post placement is a reading of the figure."""
    N = 4
    sig = np.full((N, N), 0.005)
    np.fill_diagonal(sig, 0.0)
    for a, b in ((0, 2), (0, 3), (1, 2), (1, 3)):
        sig[a, b] = sig[b, a] = 0.01
    tau = 3.0 * np.array([2.0 / 300.0, 0.1, 2.0 / 3.0, 2.0 / 3.0]) + 0.5
    x, y, z = _coords(nx, ny, 1)
    h, nstripe, R = 15.0, 8, 60.0
    width = nx / nstripe
    lub = tanh_step(h - 0.5 - y)                                    # lubricant layer
    stripe = (np.floor((x + 0.5) / width).astype(int) % 2 == 0)
    xc = nx / 2.0 - 0.5
    drop = (1.0 - lub) * tanh_step(R - np.hypot(x - xc, y - (h - 0.5)))
    C = np.zeros((N, 1, ny, nx))
    C[2] = lub * stripe
    C[3] = lub * (~stripe)
    C[1] = drop
    C[0] = np.maximum(1.0 - C[1] - C[2] - C[3], 0.0)
    C /= C.sum(axis=0, keepdims=True)
    node = np.zeros((1, ny, nx), dtype=np.uint8)
    for k in range(nstripe):
        x0 = int(round(k * width)) - 1
        for dx in range(2):
            node[0, 0:5, (x0 + dx) % nx] = SOLID
    p = base_params(D2Q9, nx, ny, 1, N, sig, tau, walls=(False, True, False), lambda_trt=3.0 / 16.0, m=m,
                    omega_stab=1.0 / 90.0, name=f"pals_{nx}x{ny}")
    p["C0"] = C
    p["geometry"] = dict(node=node, inlets=np.zeros((0, 2 + N)), outflow=False)
    p["component_force"] = (float(force), 0.0, 0.0)
    p["component_force_index"] = 1
    return p


def emulsion_2d(nx=600, ny=140, m=1.0 / 50.0):
    """The emulsion generator of Sec. V (Fig. of the microfluidic design), N = 4, built from the
    dimensions the paper lists; the figure itself is not reproduced, so the placement below is a
    reading of it.  Fluids 1..4 are components 0..3.
      - inlets of fluids 3 and 4 on the left edge: channels of width 10 and length 30 whose
        inner edges lie 55 sites from the bottom and top edges, velocity 0.003;
      - a channel of height 80 (centred) and length 30 after them, with inlets of fluid 2 of
        width 8 in its bottom and top walls right at its start, velocity 0.0045;
      - inlets of fluid 1 of width 51 in the bottom and top walls of the channel of height 110
        (centred) that follows, velocity 0.0098; it runs to the convective outflow at x = nx - 1.
    sigma_13 = sigma_14 = 0.012, the others 0.005, Omega = 1/18, eta_i = 1/12 (tau = 0.75).
    The fluid region starts as fluid 1, the two left channels as fluids 3 and 4."""
    N = 4
    sig = np.full((N, N), 0.005)
    np.fill_diagonal(sig, 0.0)
    sig[0, 2] = sig[2, 0] = sig[0, 3] = sig[3, 0] = 0.012
    node = np.full((1, ny, nx), SOLID, dtype=np.uint8)
    L1, w1, H2, H3, L2, w2, w3, H4 = 30, 10, 55, 80, 30, 8, 51, 110
    lo3 = (H2, H2 + w1)                           # fluid-3 channel rows
    lo4 = (ny - H2 - w1, ny - H2)                 # fluid-4 channel rows
    node[:, lo3[0]:lo3[1], 1:L1] = FLUID
    node[:, lo4[0]:lo4[1], 1:L1] = FLUID
    node[:, lo3[0]:lo3[1], 0] = INLET0            # inlet 0: fluid 3
    node[:, lo4[0]:lo4[1], 0] = INLET0 + 1        # inlet 1: fluid 4
    y3 = ((ny - H3) // 2, (ny + H3) // 2)
    node[:, y3[0]:y3[1], L1:L1 + L2] = FLUID
    node[:, y3[0] - 1, L1:L1 + w2] = INLET0 + 2   # inlet 2: fluid 2 from below
    node[:, y3[1], L1:L1 + w2] = INLET0 + 3       # inlet 3: fluid 2 from above
    y4 = ((ny - H4) // 2, (ny + H4) // 2)
    x4 = L1 + L2
    node[:, y4[0]:y4[1], x4:] = FLUID
    node[:, y4[0] - 1, x4:x4 + w3] = INLET0 + 4   # inlet 4: fluid 1 from below
    node[:, y4[1], x4:x4 + w3] = INLET0 + 5       # inlet 5: fluid 1 from above
    pure = np.eye(N)
    inlets = np.array([[0.003, 0.0, *pure[2]], [0.003, 0.0, *pure[3]],
                       [0.0, 0.0045, *pure[1]], [0.0, -0.0045, *pure[1]],
                       [0.0, 0.0098, *pure[0]], [0.0, -0.0098, *pure[0]]])
    C = np.zeros((N, 1, ny, nx))
    C[0] = 1.0
    for rows, comp in ((lo3, 2), (lo4, 3)):
        C[:, :, rows[0]:rows[1], :L1] = 0.0
        C[comp, :, rows[0]:rows[1], :L1] = 1.0
    p = base_params(D2Q9, nx, ny, 1, N, sig, 0.75, m=m, omega_stab=1.0 / 18.0, name=f"emulsion_{nx}x{ny}")
    p["C0"] = C
    p["geometry"] = dict(node=node, inlets=inlets, outflow=True)
    return p


def batch_sweep(nsims=512, seed=1005, sizes=(64, 96, 128, 192, 256), Ns=(3, 4, 5)):
    """Parameter sweep: even-indexed simulations are lenses, odd-indexed are Janus drops.

    Grid edge, N and the surface tensions are drawn per simulation from the
    generator seeded with seed + index.  All are FP32-path jobs with tau = 1.
    """
    sims = []
    for s in range(nsims):
        rng = np.random.default_rng(seed + s)
        n = int(rng.choice(sizes))
        N = int(rng.choice(Ns))
        sig = random_sigma(rng, N)
        if s % 2 == 0:
            p = lens_2d(nx=n, ny=n, radius=n * 12.0 / 64.0,
                        sigma3=(sig[0, 1], sig[0, 2], sig[1, 2]), tau=1.0, m=0.05,
                        extra_sigma=sig, N=N, walls_y=True)
        else:
            x, y, z = _coords(n, n, 1)
            c = n / 2.0 - 0.5
            rad = n * 20.0 / 100.0
            drop = tanh_step(rad - np.hypot(x - c, y - c))
            h = tanh_step(x - c)
            C = np.zeros((N, 1, n, n))
            C[1] = drop * (1.0 - h)
            C[2] = drop * h
            for e in range(3, N):
                cx = (e - 2) * n / (N - 1) - 0.5
                d = tanh_step(n / 8.0 - np.hypot(x - cx, y - (n / 8.0 + 1.5)))
                C[1:e] *= (1.0 - d)
                C[e] = d
            C[0] = 1.0 - C[1:].sum(axis=0)
            p = base_params(D2Q9, n, n, 1, N, sig, 1.0, m=0.05, name=f"janus_{n}_N{N}")
            p["C0"] = C
        p["index"] = s
        sims.append(p)
    return sims


# The five reference workloads, by name; each entry builds its parameter dict.
CONFIGS = {
    "lens64_N3_fp64": lambda: lens_2d(),
    "spinodal512_N4": lambda: spinodal_2d(),
    "poiseuille3d_N7": lambda: layered_poiseuille(),
    "janus3d256_N4": lambda: janus_3d(),
}
