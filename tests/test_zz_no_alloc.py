"""The allocation-free plaquette entry point against the handle-based one.

su2_plaquette_static serves callers that cannot allocate device memory: it
reads a caller-owned link store and keeps its reduction scratch in a fixed
array inside the library.  This file sorts last so that a run stopping at the
first failure has already run every other test; it passes both alone in a
fresh process and after the rest of the suite.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1010_4834_gb300 import Lattice, _lib

pytestmark = pytest.mark.gpu

# same tolerances as the other measurement parity tests
MTOL = {"f64": 1e-12, "f32": 2e-6, "f16q": 2e-3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def static_plaquette(lat):
    import torch
    L = _lib.load()
    out = np.full(3, np.nan)
    stream = C.c_void_p(int(torch.cuda.current_stream().cuda_stream) or 1)
    rc = L.su2_plaquette_static(C.c_void_p(lat._buf.data_ptr()), _lib.dims_arg(lat.dims), lat.prec,
                                out.ctypes.data_as(C.POINTER(C.c_double)), stream)
    assert rc == 0, L.su2_last_error()
    return out


@pytest.mark.parametrize("prec,dims", [(p, d) for p in ("f64", "f32", "f16q") for d in ((8, 8, 8, 8), (6, 4, 2, 10))]
                         # 32^4 needs 4096 blocks of 256 sites: the grid is capped at the
                         # device's occupancy, so the grid-stride loop and the last block's
                         # sum over more than 256 partials both run
                         + [("f32", (32, 32, 32, 32))])
def test_static_scratch_plaquette_matches(dims, prec):
    lat = Lattice(dims, 2.4, seed=3, start="hot", prec=prec)
    lat.sweep(2)
    for _ in range(2):                       # two calls in a row share the fixed scratch
        ref = lat.plaquette()
        got = static_plaquette(lat)
        np.testing.assert_allclose(got, ref, atol=MTOL[prec], rtol=0)
        assert np.abs(got - static_plaquette(lat)).max() == 0.0
        # and against the oracle's plaquette of the same links
        np.testing.assert_allclose(got, oracle.plaquette(list(dims), lat.get_links()), atol=MTOL[prec], rtol=0)
        lat.sweep(1)                         # a different configuration for the next call
    lat.close()


def test_static_plaquette_allocates_no_device_memory():
    # after a first call (which looks the fixed array up), further calls leave
    # the device's free memory exactly as it was
    import torch
    lat = Lattice((16, 16, 16, 16), 2.4, seed=5, start="hot", prec="f32")
    first = static_plaquette(lat)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(10):
        np.testing.assert_array_equal(static_plaquette(lat), first)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    lat.close()


def test_static_plaquette_rejects_bad_arguments():
    L = _lib.load()
    out = np.empty(3)
    lat = Lattice((4, 4, 4, 4), 2.0, prec="f32")
    ptr = C.c_void_p(lat._buf.data_ptr())
    dp = out.ctypes.data_as(C.POINTER(C.c_double))
    assert L.su2_plaquette_static(ptr, _lib.dims_arg((4, 4, 4, 5)), _lib.F32, dp, None) == _lib.EINVAL
    assert L.su2_plaquette_static(ptr, _lib.dims_arg((4, 4, 4, 4)), 9, dp, None) == _lib.EINVAL
    assert L.su2_plaquette_static(None, _lib.dims_arg((4, 4, 4, 4)), _lib.F32, dp, None) == _lib.EINVAL
    lat.close()
