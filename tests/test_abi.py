"""The C ABI without a GPU: the library builds, loads and exports every declared
symbol; argument validation and the host-side Sec. II tables work on the CPU."""
import math
import re
import os

import numpy as np
import pytest

import nfe_workloads as W
import paper_2605_22214_gb300 as nfe
from oracle import thermo

from ._lib import lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(nfe_\w+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported():
    L = lib()
    declared = _declared()
    assert declared, "no declarations found"
    assert declared == set(nfe.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


def _params(N=3, **kw):
    sig = np.full((N, N), 0.005)
    np.fill_diagonal(sig, 0)
    p = W.base_params(9, 8, 8, 1, N, sig, 1.0)
    p.update(kw)
    return p


@pytest.mark.parametrize("bad,status", [
    (dict(N=1), 1), (dict(N=9), 1), (dict(nz=2), 1), (dict(nx=0), 1),
    (dict(tau=np.array([0.5, 1.0, 1.0])), 1), (dict(D=0.0), 1), (dict(implicit=3), 1),
])
def test_create_rejects_bad_arguments_before_touching_the_gpu(bad, status):
    lib()
    p = _params()
    N = bad.pop("N", 3)
    p.update(bad)
    if N != 3:
        sig = np.full((N, N), 0.005)
        np.fill_diagonal(sig, 0)
        p["sigma"], p["tau"], p["N"] = sig, np.ones(N), N
    with pytest.raises(nfe.NfeError) as e:
        nfe.Sim(p)
    assert e.value.status == status


def test_tau_g_validation():
    # tau_g must exceed 1/2 (0 selects 1); tau_g != 1 does not combine with NO_PHI.
    lib()
    p = _params(tau_g=0.5)
    with pytest.raises(nfe.NfeError) as e:
        nfe.Sim(p)
    assert e.value.status == 1          # NFE_EINVAL
    with pytest.raises(nfe.NfeError) as e:
        nfe.Sim(_params(tau_g=1.3), flags=nfe.NFE_NO_PHI)
    assert e.value.status == 7


def test_create_rejects_bad_sigma():
    lib()
    p = _params()
    p["sigma"] = p["sigma"].copy()
    p["sigma"][0, 1] = 0.006          # not symmetric
    with pytest.raises(nfe.NfeError):
        nfe.Sim(p)
    p = _params()
    p["sigma"] = p["sigma"].copy()
    p["sigma"][0, 0] = 0.001          # non-zero diagonal
    with pytest.raises(nfe.NfeError):
        nfe.Sim(p)


def test_status_strings():
    lib()
    for s in range(8):
        assert nfe.nfe_status_string(s)


@pytest.mark.parametrize("N,imp", [(3, 2), (4, 0), (5, 4), (6, 1), (7, 6), (8, 3)])
def test_library_stabiliser_part_matches_oracle(N, imp):
    # The quartic (Omega) part of the library's flux potential alone, S(Omega) - S(0), against
    # the oracle's literal xi_j (Eqs. 17-19): the library stores it in a structured form
    # (squared pair products times linear forms), so this checks that form term by term.
    lib()
    rng = np.random.default_rng(80 + N)
    sig = W.random_sigma(rng, N)
    pts = W.random_simplex_points(rng, N, 200)
    om = 1.0 / 90.0
    d_lib = (nfe.nfe_bulk_potential_host(sig, pts, omega_stab=om, implicit=imp)
             - nfe.nfe_bulk_potential_host(sig, pts, omega_stab=0.0, implicit=imp))
    d_or = (thermo.Tables(sig, omega=om).bulk_flux_potential(pts.T).T
            - thermo.Tables(sig, omega=0.0).bulk_flux_potential(pts.T).T)
    ev = [c for c in range(N) if c != imp]
    scale = np.abs(d_or[:, ev]).max()
    assert scale > 0.0
    np.testing.assert_allclose(d_lib[:, ev], d_or[:, ev], rtol=0, atol=1e-10 * scale)


@pytest.mark.parametrize("N,omega,imp", [(2, 0.0, 1), (3, 0.0, 0), (4, 0.0, 3), (4, 1 / 90, 1),
                                         (5, float("nan"), 2), (6, 0.0, 5), (7, 1 / 90, 0), (8, 0.0, 4)])
def test_library_tables_match_oracle(N, omega, imp):
    # The library's own Sec. II tables (C++, independent of the oracle) give the same bulk
    # flux potential as the oracle's literal Eq. 12 on the simplex, and exactly 0 for an
    # absent evolved component.
    lib()
    rng = np.random.default_rng(50 + N)
    sig = W.random_sigma(rng, N)
    T = thermo.Tables(sig, omega=omega)
    pts = W.random_simplex_points(rng, N, 200)
    S_lib = nfe.nfe_bulk_potential_host(sig, pts, omega_stab=omega, implicit=imp)
    S_or = T.bulk_flux_potential(pts.T).T
    ev = [c for c in range(N) if c != imp]
    np.testing.assert_allclose(S_lib[:, ev], S_or[:, ev], rtol=0, atol=1e-12 * np.abs(S_or).max())
    absent = ev[-1]
    pts0 = W.random_simplex_points(rng, N, 50, absent=absent)
    assert (nfe.nfe_bulk_potential_host(sig, pts0, omega_stab=omega, implicit=imp)[:, absent] == 0.0).all()


def test_struct_layouts_match_the_header(tmp_path):
    # sizes and field offsets of every public struct, from the C compiler against the ctypes mirror
    import ctypes
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    structs = {"nfe_grid": nfe.nfe_grid, "nfe_params": nfe.nfe_params, "nfe_diag": nfe.nfe_diag,
               "nfe_info": nfe.nfe_info}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "nfe.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name}.{field} %zu\\n", offsetof({name}, {field}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run(["gcc", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                      text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert int(got[f"{name}.{field}"]) == getattr(cls, field).offset, (name, field)
