"""The allocation-free statistics entry point against nfe_diagnostics.

nfe_field_stats_static serves callers that cannot allocate device memory (code
inside another runtime's pool or a fixed arena): its partial sums live in a
static device array of the library.  This test feeds it the fields of a running
simulation (copied to device memory the test owns) and compares its sums,
largest magnitudes and minima with what nfe_diagnostics reports for the same
state, on two calls in a row with different data.  It sits in a file of its own
so that pytest collects it last.
"""
import numpy as np
import pytest

import nfe_workloads as W
import paper_2605_22214_gb300 as nfe

from ._lib import lib

pytestmark = pytest.mark.gpu


def _stats_on_device(planes):
    import torch
    d_planes = torch.tensor(np.ascontiguousarray(planes), dtype=torch.float64, device="cuda")
    d_out = torch.full((planes.shape[0], 4), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    nfe.nfe_field_stats_static(planes.shape[0], planes.shape[1], d_planes.data_ptr(), d_out.data_ptr(), None)
    torch.cuda.synchronize()
    return d_out.cpu().numpy()


def test_static_stats_match_diagnostics_on_two_calls():
    lib()
    p = W.spinodal_2d(nx=96, ny=80, seed=21)
    N = p["N"]
    with nfe.Sim(p, "fp64") as s:
        s.set_fields(p["C0"])
        for steps in (20, 35):                       # two calls in a row, different states
            s.step(steps)
            d = s.diagnostics()
            C, v, P = s.fields()
            planes = np.concatenate([C.reshape(N, -1), v.reshape(3, -1)])
            out = _stats_on_device(planes)
            # FP64 sums in another order: 1e-12 relative, as for the FP64 fields
            np.testing.assert_allclose(out[:N, 0], d["mass"], rtol=1e-12)
            np.testing.assert_allclose(out[:N, 2], d["max_abs_C"], rtol=1e-12)
            np.testing.assert_allclose(out[:N, 3], d["min_C"], rtol=1e-12)
            scale = out[N:, 1].sum()
            np.testing.assert_allclose(out[N:, 0], d["momentum"], rtol=0, atol=1e-12 * scale + 1e-300)
            # host reference for the remaining statistic (sum of |.|)
            np.testing.assert_allclose(out[:, 1], np.abs(planes).sum(axis=1), rtol=1e-12)


def test_static_stats_reject_too_many_planes():
    import torch
    lib()
    buf = torch.zeros(17 * 10, dtype=torch.float64, device="cuda")
    out = torch.zeros(17 * 4, dtype=torch.float64, device="cuda")
    with pytest.raises(nfe.NfeError) as e:
        nfe.nfe_field_stats_static(17, 10, buf.data_ptr(), out.data_ptr(), None)
    assert e.value.status == 1
    assert "16" in str(e.value)


def test_static_stats_report_a_nan():
    # a NaN anywhere in a plane shows in every statistic of that plane (a health check on the
    # largest magnitude must not miss it); the other planes are unaffected
    lib()
    planes = np.linspace(-1.0, 2.0, 3 * 1000).reshape(3, 1000)
    planes[1, 617] = np.nan
    out = _stats_on_device(planes)
    assert np.isnan(out[1]).all()
    np.testing.assert_allclose(out[[0, 2], 2], np.abs(planes[[0, 2]]).max(axis=1), rtol=0)
    np.testing.assert_allclose(out[[0, 2], 3], planes[[0, 2]].min(axis=1), rtol=0)
