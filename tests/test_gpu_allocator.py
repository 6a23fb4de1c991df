"""Device memory through the caller's allocator hooks (nfe_params.device_alloc / device_free):
PyTorch's caching allocator holds every state buffer of a simulation, the results are bit for
bit those of cudaMalloc buffers, and everything is given back at destroy."""
import numpy as np
import pytest

import nfe_workloads as W
import paper_2605_22214_gb300 as nfe

from ._lib import lib

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    lib()


def _run(p, **kw):
    with nfe.Sim(p, "fp32", **kw) as s:
        s.set_fields(p["C0"])
        s.step(10)
        s.sync()
        s.diagnostics()
        return s.get_state(), s.info()["device_bytes"]


def test_torch_caching_allocator_holds_the_simulation():
    torch = pytest.importorskip("torch")
    p = W.spinodal_2d(nx=96, ny=64, seed=5)
    base = torch.cuda.memory_allocated()
    with nfe.Sim(p, "fp32", allocator="torch") as s:
        assert torch.cuda.memory_allocated() - base >= s.info()["device_bytes"] > 0
    assert torch.cuda.memory_allocated() == base
    hooked, nbytes = _run(p, allocator="torch")
    assert torch.cuda.memory_allocated() == base
    plain, nbytes2 = _run(p)
    assert np.array_equal(hooked, plain) and nbytes == nbytes2


def test_allocator_failure_is_reported():
    p = W.spinodal_2d(nx=32, ny=32, seed=6)
    calls = []

    def alloc(nbytes):
        calls.append(nbytes)
        return 0                      # refuse every request

    with pytest.raises(nfe.NfeError) as e:
        nfe.Sim(p, "fp32", allocator=(alloc, lambda ptr: None))
    assert e.value.status == 2 and calls
