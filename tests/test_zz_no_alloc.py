"""fdirw_mass_noalloc: the mass budget for callers that may not allocate device memory.

Such callers (a framework that owns all device memory, a real-time loop that must not allocate, code with
no fdirw context) get the FP64 total of a device field from a fixed scratch array inside the library.
This file is collected last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2408_11376_gb300 import FDiRW, FdirwError, fdirw, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    from paper_2408_11376_gb300 import build
    build.build()                      # no-op when libfdirw.so is up to date


def test_mass_noalloc_matches_fdirw_mass_on_consecutive_calls():
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    shape = (70, 64, 50)                                   # 224,000 cells: 4 scratch chunks, ragged tail
    n = int(np.prod(shape))
    fields = [torch.from_numpy(synth.random_field(n, 1, 0.0, 3.0)).to(dev),
              torch.from_numpy(synth.random_field(n, 2, -1.0, 1.0)).to(dev)]
    D = torch.ones(n, dtype=torch.float64, device=dev)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=dev)
    with FDiRW(shape, D, 0.1, 1, 1) as f:                  # the existing entry point, for comparison
        expected = [f.mass(c) for c in fields]
    for c, m in zip(fields, expected):                      # two calls in a row, same scratch
        fdirw.fdirw_mass_noalloc(c, out)
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - m) <= 1e-12 * max(1.0, abs(m)), (got, m)
    # a call on a smaller field after a larger one: stale partials beyond its chunks are never read
    small = fields[0][: 1000]
    fdirw.fdirw_mass_noalloc(small, out)
    torch.cuda.synchronize()
    assert abs(float(out.item()) - float(small.sum().item())) <= 1e-12 * float(small.sum().item())
    # an empty field: only the final kernel runs, and it writes 0
    fdirw.fdirw_mass_noalloc(fields[0][:0], out)
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0


def test_mass_noalloc_rejects_what_it_cannot_serve():
    dev = torch.device("cuda:0")
    c = torch.ones(16, dtype=torch.float64, device=dev)
    out = torch.zeros(1, dtype=torch.float64, device=dev)
    lib = fdirw.load()
    import ctypes
    rc = lib.fdirw_mass_noalloc(ctypes.c_void_p(c.data_ptr()), (1 << 30) + 1, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == fdirw.FDIRW_ERR_ARG and "2^30" in fdirw.fdirw_last_error()
    host = np.ones(16)
    with pytest.raises(FdirwError):
        fdirw.fdirw_mass_noalloc(host, out)                 # host memory is not accepted
