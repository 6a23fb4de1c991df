"""Python binding of libnfe (include/nfe.h): argument marshalling only.

Every step of the lattice update runs in the CUDA kernels behind the C ABI;
this module converts numpy arrays and dicts to the C structs and back.  It
loads `libnfe.so` from this package directory and raises if the library is
missing (build it with `paper_2605_22214_gb300.build.build()`): there is no
other implementation to fall back to.

The functions carry the C names (`nfe_create`, `nfe_step`, ...); `Sim` wraps
one simulation handle.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libnfe.so")

NFE_D2Q9, NFE_D3Q19 = 9, 19
NFE_FP64, NFE_FP32, NFE_FP32_F16STORE, NFE_FP32_BF16STORE = 0, 1, 2, 3
NFE_WALL_X, NFE_WALL_Y, NFE_WALL_Z = 1, 2, 4
NFE_NONCONSERVATIVE_FORCE, NFE_NO_PHI = 1, 2
NFE_MAX_N = 8
PRECISIONS = {"fp64": NFE_FP64, "fp32": NFE_FP32, "f16": NFE_FP32_F16STORE, "bf16": NFE_FP32_BF16STORE}
STATUS = {0: "NFE_OK", 1: "NFE_EINVAL", 2: "NFE_ENOMEM", 3: "NFE_ECUDA", 4: "NFE_ESINGULAR",
          5: "NFE_ENONFINITE", 6: "NFE_ETIMEOUT", 7: "NFE_EUNSUPPORTED"}

# every symbol include/nfe.h declares
EXPORTS = ["nfe_create", "nfe_set_fields", "nfe_step", "nfe_sync", "nfe_fields", "nfe_populations",
           "nfe_diagnostics", "nfe_domain_size", "nfe_get_state", "nfe_set_state", "nfe_get_info", "nfe_profile_enable",
           "nfe_profile_read", "nfe_destroy", "nfe_status_string", "nfe_last_error",
           "nfe_bulk_potential_host", "nfe_set_variant", "nfe_field_stats_static", "nfe_set_geometry",
           "nfe_batch_create", "nfe_batch_set_fields", "nfe_batch_step", "nfe_batch_set_mode",
           "nfe_batch_sync", "nfe_batch_fields", "nfe_batch_diagnostics", "nfe_batch_get_info",
           "nfe_batch_set_barrier_test", "nfe_batch_destroy"]
NFE_BATCH_PERSISTENT, NFE_BATCH_PER_STEP, NFE_BATCH_AUTO = 0, 1, 2


class nfe_grid(C.Structure):
    _fields_ = [("lattice", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("wall_mask", C.c_uint)]


# device memory hooks (nfe_alloc_fn / nfe_free_fn)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class nfe_params(C.Structure):
    _fields_ = [("sigma", C.POINTER(C.c_double)), ("tau", C.POINTER(C.c_double)),
                ("lambda_trt", C.c_double), ("m", C.c_double), ("D", C.c_double),
                ("omega_stab", C.c_double), ("body_force", C.c_double * 3),
                ("precision", C.c_int), ("implicit_component", C.c_int), ("flags", C.c_int),
                ("scale_exp", C.c_int), ("cuda_stream", C.c_void_p), ("tau_g", C.c_double),
                ("component_force", C.c_double * 3), ("component_force_index", C.c_int),
                ("device_alloc", ALLOC_FN), ("device_free", FREE_FN), ("alloc_ctx", C.c_void_p)]


class nfe_diag(C.Structure):
    _fields_ = [("step", C.c_int64), ("N", C.c_int), ("mass", C.c_double * NFE_MAX_N),
                ("momentum", C.c_double * 3), ("force_sum", C.c_double * 3),
                ("force_abs_sum", C.c_double * 3), ("max_abs_C", C.c_double * NFE_MAX_N),
                ("min_C", C.c_double * NFE_MAX_N), ("max_speed", C.c_double), ("nonfinite", C.c_int)]


class nfe_info(C.Structure):
    _fields_ = [("lattice", C.c_int), ("N", C.c_int), ("precision", C.c_int), ("sites", C.c_int64),
                ("omega_stab", C.c_double), ("factor_residual", C.c_double),
                ("kernels_per_step", C.c_int), ("variant", C.c_int), ("nvariants", C.c_int),
                ("min_bytes_per_site", C.c_double),
                ("state_bytes", C.c_size_t), ("device_bytes", C.c_size_t)]


class nfe_batch_info(C.Structure):
    _fields_ = [("nsims", C.c_int), ("sites", C.c_int64), ("nitems", C.c_int), ("grid", C.c_int),
                ("tile_x", C.c_int), ("tile_y", C.c_int), ("graphs", C.c_int), ("form", C.c_int)]


class NfeError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None


def load():
    """Load libnfe.so (once); raises if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: the CUDA library must be built "
                          "(paper_2605_22214_gb300.build.build()); there is no fallback path")
    lib = C.CDLL(LIB_PATH)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    sig = {
        "nfe_create": ([C.POINTER(nfe_grid), C.c_int, C.POINTER(nfe_params), C.POINTER(P)], C.c_int),
        "nfe_set_fields": ([P, dp, dp], C.c_int),
        "nfe_step": ([P, C.c_int64], C.c_int),
        "nfe_sync": ([P], C.c_int),
        "nfe_fields": ([P, dp, dp, dp], C.c_int),
        "nfe_populations": ([P, dp], C.c_int),
        "nfe_diagnostics": ([P, C.POINTER(nfe_diag)], C.c_int),
        "nfe_domain_size": ([P, dp, C.c_int, C.c_int, dp], C.c_int),
        "nfe_get_state": ([P, P, C.c_size_t], C.c_int),
        "nfe_set_state": ([P, P, C.c_size_t], C.c_int),
        "nfe_get_info": ([P, C.POINTER(nfe_info)], C.c_int),
        "nfe_profile_enable": ([P, C.c_int], C.c_int),
        "nfe_set_variant": ([P, C.c_int], C.c_int),
        "nfe_set_geometry": ([P, C.c_void_p, C.c_int, dp, C.c_int], C.c_int),
        "nfe_field_stats_static": ([C.c_int, C.c_int64, P, P, P], C.c_int),
        "nfe_batch_create": ([C.c_int, C.POINTER(nfe_grid), C.POINTER(C.c_int), C.POINTER(nfe_params),
                              C.POINTER(P)], C.c_int),
        "nfe_batch_set_fields": ([P, C.c_int, dp, dp], C.c_int),
        "nfe_batch_step": ([P, C.c_int64], C.c_int),
        "nfe_batch_set_mode": ([P, C.c_int], C.c_int),
        "nfe_batch_sync": ([P], C.c_int),
        "nfe_batch_fields": ([P, C.c_int, dp, dp, dp], C.c_int),
        "nfe_batch_diagnostics": ([P, C.c_int, C.POINTER(nfe_diag)], C.c_int),
        "nfe_batch_get_info": ([P, C.POINTER(nfe_batch_info)], C.c_int),
        "nfe_batch_set_barrier_test": ([P, C.c_int64, C.c_int], C.c_int),
        "nfe_batch_destroy": ([P], None),
        "nfe_profile_read": ([P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_char_p),
                              C.POINTER(C.c_int64), dp], C.c_int),
        "nfe_destroy": ([P], None),
        "nfe_status_string": ([C.c_int], C.c_char_p),
        "nfe_last_error": ([], C.c_char_p),
        "nfe_bulk_potential_host": ([C.c_int, dp, C.c_double, C.c_double, C.c_int, C.c_int, dp, dp], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(status):
    if status != 0:
        raise NfeError(status, load().nfe_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


# -- functions with the C names -------------------------------------------------

def make_grid(p):
    walls = p.get("walls", (False, False, False))
    mask = (NFE_WALL_X if walls[0] else 0) | (NFE_WALL_Y if walls[1] else 0) | (NFE_WALL_Z if walls[2] else 0)
    return nfe_grid(int(p["lattice"]), int(p["nx"]), int(p["ny"]), int(p["nz"]), mask)


def make_params(p, precision="fp64", stream=None, flags=0, scale_exp=0):
    """nfe_params from a parameter dict (the `nfe_workloads` layout); keeps the arrays alive."""
    N = int(p["N"])
    sigma = np.ascontiguousarray(np.asarray(p["sigma"], dtype=np.float64).reshape(N, N))
    tau = np.ascontiguousarray(np.asarray(p["tau"], dtype=np.float64).reshape(N))
    prm = nfe_params()
    prm.sigma = _dptr(sigma)
    prm.tau = _dptr(tau)
    prm.lambda_trt = float(p.get("lambda_trt", -1.0))
    prm.m = float(p["m"])
    prm.D = float(p.get("D", 4.0))
    prm.omega_stab = float(p.get("omega_stab", math.nan))
    prm.body_force = (C.c_double * 3)(*[float(b) for b in p.get("body_force", (0.0, 0.0, 0.0))])
    prm.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    prm.implicit_component = int(p.get("implicit", N - 1))
    prm.flags = int(flags)
    prm.scale_exp = int(scale_exp)
    prm.cuda_stream = stream
    prm.tau_g = float(p.get("tau_g", 1.0))
    prm.component_force = (C.c_double * 3)(*[float(b) for b in p.get("component_force", (0.0, 0.0, 0.0))])
    prm.component_force_index = int(p.get("component_force_index", 0))
    prm._keep = (sigma, tau)
    return prm


def nfe_create(grid, N, params):
    h = C.c_void_p()
    _check(load().nfe_create(C.byref(grid), int(N), C.byref(params), C.byref(h)))
    return h


def nfe_set_fields(h, Cf, v=None):
    Cf = np.ascontiguousarray(Cf, dtype=np.float64)
    v = None if v is None else np.ascontiguousarray(v, dtype=np.float64)
    _check(load().nfe_set_fields(h, _dptr(Cf), _dptr(v)))


def nfe_step(h, nsteps):
    _check(load().nfe_step(h, int(nsteps)))


def nfe_sync(h):
    _check(load().nfe_sync(h))


def nfe_fields(h, N, n):
    Cf = np.empty((N, n))
    v = np.empty((3, n))
    P = np.empty(n)
    _check(load().nfe_fields(h, _dptr(Cf), _dptr(v), _dptr(P)))
    return Cf, v, P


def nfe_populations(h, Q, n):
    f = np.empty((Q - 1, n))
    _check(load().nfe_populations(h, _dptr(f)))
    return f


def nfe_diagnostics(h):
    d = nfe_diag()
    _check(load().nfe_diagnostics(h, C.byref(d)))
    N = d.N
    return dict(step=d.step, mass=np.array(d.mass[:N]), momentum=np.array(d.momentum[:]),
                force_sum=np.array(d.force_sum[:]), force_abs_sum=np.array(d.force_abs_sum[:]),
                max_abs_C=np.array(d.max_abs_C[:N]), min_C=np.array(d.min_C[:N]),
                max_speed=d.max_speed, nonfinite=d.nonfinite)


def nfe_domain_size(h, N, component=0, nbins=0):
    """(L of every component (user order), their mean, shell-averaged S(k) of `component` or None)."""
    L = np.zeros(N + 1)
    Sk = np.zeros(max(nbins, 1))
    _check(load().nfe_domain_size(h, _dptr(L), int(component), int(nbins), _dptr(Sk) if nbins > 0 else None))
    return L[:N], L[N], (Sk[:nbins] if nbins > 0 else None)


def nfe_set_geometry(h, node, inlets=None, outflow=False):
    """Node classes (uint8 per site, x fastest; None removes the geometry), inlet rows
    (vx, vy, C_1..C_N on D2Q9; vx, vy, vz, C_1..C_N on D3Q19) and the convective outflow on the
    x = nx - 1 edge."""
    if node is None:
        _check(load().nfe_set_geometry(h, None, 0, None, 0))
        return
    node = np.ascontiguousarray(node, dtype=np.uint8).ravel()
    tab = np.ascontiguousarray(np.zeros((0, 1)) if inlets is None else inlets, dtype=np.float64)
    k = tab.shape[0] if tab.size else 0
    _check(load().nfe_set_geometry(h, node.ctypes.data_as(C.c_void_p), k, _dptr(tab.ravel()) if k else None,
                                   1 if outflow else 0))


def nfe_get_info(h):
    i = nfe_info()
    _check(load().nfe_get_info(h, C.byref(i)))
    return {name: getattr(i, name) for name, _ in nfe_info._fields_}


def nfe_get_state(h, out=None):
    nbytes = nfe_get_info(h)["state_bytes"]
    buf = np.empty(nbytes, dtype=np.uint8) if out is None else out
    _check(load().nfe_get_state(h, buf.ctypes.data_as(C.c_void_p), nbytes))
    return buf


def nfe_set_state(h, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(load().nfe_set_state(h, buf.ctypes.data_as(C.c_void_p), buf.nbytes))


def nfe_get_state_ptr(h, ptr, nbytes):
    """Raw-pointer form (e.g. pinned host memory from torch)."""
    _check(load().nfe_get_state(h, C.c_void_p(ptr), int(nbytes)))


def nfe_set_state_ptr(h, ptr, nbytes):
    _check(load().nfe_set_state(h, C.c_void_p(ptr), int(nbytes)))


def nfe_set_variant(h, variant):
    _check(load().nfe_set_variant(h, int(variant)))


def nfe_profile_enable(h, on=True):
    _check(load().nfe_profile_enable(h, 1 if on else 0))


def nfe_profile_read(h):
    kinds = C.c_int()
    names = (C.c_char_p * 8)()
    launches = (C.c_int64 * 8)()
    ms = (C.c_double * 8)()
    _check(load().nfe_profile_read(h, 8, C.byref(kinds), names, launches, ms))
    return {names[i].decode(): (launches[i], ms[i]) for i in range(kinds.value)}


def nfe_destroy(h):
    if h:
        load().nfe_destroy(h)


def nfe_field_stats_static(nplanes, n, d_planes_ptr, d_out_ptr, stream=None):
    """Allocation-free FP64 sum / sum|.| / max|.| / min of device planes (raw device pointers)."""
    _check(load().nfe_field_stats_static(int(nplanes), int(n), C.c_void_p(d_planes_ptr),
                                         C.c_void_p(d_out_ptr), stream))


def nfe_status_string(status):
    return load().nfe_status_string(int(status)).decode()


def nfe_last_error():
    return load().nfe_last_error().decode()


def nfe_bulk_potential_host(sigma, C_pts, D=4.0, omega_stab=math.nan, implicit=None):
    """Library's factored bulk flux potential at host points C_pts (npts x N); host only."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    N = sigma.shape[0]
    pts = np.ascontiguousarray(C_pts, dtype=np.float64).reshape(-1, N)
    S = np.empty_like(pts)
    _check(load().nfe_bulk_potential_host(N, _dptr(sigma), float(D), float(omega_stab),
                                          N - 1 if implicit is None else int(implicit),
                                          pts.shape[0], _dptr(pts), _dptr(S)))
    return S


def _allocator_hooks(allocator, stream):
    if allocator == "torch":
        import torch
        tstream = torch.cuda.ExternalStream(stream) if stream else None
        dev = torch.cuda.current_device()

        def alloc(nbytes):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev, stream=tstream)
            except RuntimeError:
                return 0

        def free(ptr):
            torch.cuda.caching_allocator_delete(ptr)
    else:
        alloc, free = allocator
    return (ALLOC_FN(lambda nbytes, ctx: alloc(nbytes) or None),
            FREE_FN(lambda ptr, ctx: free(ptr)))


class Sim:
    """One simulation on cuda:0 (owns an nfe_sim handle)."""

    def __init__(self, p, precision="fp64", stream=None, flags=0, scale_exp=0, allocator=None):
        self.p = p
        self.N = int(p["N"])
        self.Q = int(p["lattice"])
        self.n = int(p["nx"]) * int(p["ny"]) * int(p["nz"])
        self.shape = (int(p["nz"]), int(p["ny"]), int(p["nx"]))
        self._grid = make_grid(p)
        self._params = make_params(p, precision, stream, flags, scale_exp)
        # allocator: None (cudaMalloc), "torch" (PyTorch's caching allocator), or a pair of
        # callables (alloc(bytes) -> int pointer or 0, free(pointer)); the callbacks live as
        # long as this object
        self._hooks = None
        if allocator is not None:
            self._hooks = _allocator_hooks(allocator, stream)
            self._params.device_alloc, self._params.device_free = self._hooks
        self.h = nfe_create(self._grid, self.N, self._params)

    def set_fields(self, Cf, v=None):
        nfe_set_fields(self.h, np.asarray(Cf).reshape(self.N, self.n),
                       None if v is None else np.asarray(v).reshape(3, self.n))

    def step(self, nsteps=1):
        nfe_step(self.h, nsteps)

    def sync(self):
        nfe_sync(self.h)

    def fields(self):
        Cf, v, P = nfe_fields(self.h, self.N, self.n)
        return (Cf.reshape((self.N,) + self.shape), v.reshape((3,) + self.shape), P.reshape(self.shape))

    def populations(self):
        return nfe_populations(self.h, self.Q, self.n).reshape((self.Q - 1,) + self.shape)

    def diagnostics(self):
        return nfe_diagnostics(self.h)

    def domain_size(self, component=0, nbins=0):
        return nfe_domain_size(self.h, self.N, component, nbins)

    def info(self):
        return nfe_get_info(self.h)

    def get_state(self):
        return nfe_get_state(self.h)

    def set_state(self, buf):
        nfe_set_state(self.h, buf)

    def set_variant(self, variant):
        nfe_set_variant(self.h, variant)

    def set_geometry(self, node, inlets=None, outflow=False):
        nfe_set_geometry(self.h, node, inlets, outflow)

    def profile_enable(self, on=True):
        nfe_profile_enable(self.h, on)

    def profile_read(self):
        return nfe_profile_read(self.h)

    def close(self):
        if self.h:
            nfe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Many independent D2Q9 simulations advanced together (per-step launches or one persistent
    launch); a member's dict may carry "flags" and "tau_g"."""

    def __init__(self, plist, precision="fp32", stream=None):
        self.plist = list(plist)
        n = len(self.plist)
        grids = (nfe_grid * n)(*[make_grid(p) for p in self.plist])
        Ns = (C.c_int * n)(*[int(p["N"]) for p in self.plist])
        # per-member flags (NFE_NO_PHI, NFE_NONCONSERVATIVE_FORCE) and tau_g come with its dict
        self._params = [make_params(p, precision, stream, flags=int(p.get("flags", 0))) for p in self.plist]
        params = (nfe_params * n)(*self._params)
        h = C.c_void_p()
        _check(load().nfe_batch_create(n, grids, Ns, params, C.byref(h)))
        self.h = h
        self._keep = (grids, Ns, params)

    def _size(self, i):
        p = self.plist[i]
        return int(p["N"]), int(p["nx"]) * int(p["ny"]) * int(p["nz"]), (int(p["nz"]), int(p["ny"]), int(p["nx"]))

    def set_fields(self, i, Cf, v=None):
        N, n, _ = self._size(i)
        Cf = np.ascontiguousarray(np.asarray(Cf, dtype=np.float64).reshape(N, n))
        v = None if v is None else np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(3, n))
        _check(load().nfe_batch_set_fields(self.h, int(i), _dptr(Cf), _dptr(v)))

    def step(self, nsteps=1):
        _check(load().nfe_batch_step(self.h, int(nsteps)))

    def set_mode(self, mode):
        _check(load().nfe_batch_set_mode(self.h, int(mode)))

    def sync(self):
        _check(load().nfe_batch_sync(self.h))

    def fields(self, i):
        N, n, shape = self._size(i)
        Cf, v, P = np.empty((N, n)), np.empty((3, n)), np.empty(n)
        _check(load().nfe_batch_fields(self.h, int(i), _dptr(Cf), _dptr(v), _dptr(P)))
        return Cf.reshape((N,) + shape), v.reshape((3,) + shape), P.reshape(shape)

    def diagnostics(self, i):
        d = nfe_diag()
        _check(load().nfe_batch_diagnostics(self.h, int(i), C.byref(d)))
        N = d.N
        return dict(step=d.step, mass=np.array(d.mass[:N]), momentum=np.array(d.momentum[:]),
                    force_sum=np.array(d.force_sum[:]), max_abs_C=np.array(d.max_abs_C[:N]),
                    min_C=np.array(d.min_C[:N]), max_speed=d.max_speed, nonfinite=d.nonfinite)

    def info(self):
        i = nfe_batch_info()
        _check(load().nfe_batch_get_info(self.h, C.byref(i)))
        return {name: getattr(i, name) for name, _ in nfe_batch_info._fields_}

    def set_barrier_test(self, spins, extra):
        _check(load().nfe_batch_set_barrier_test(self.h, int(spins), int(extra)))

    def close(self):
        if getattr(self, "h", None):
            load().nfe_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
