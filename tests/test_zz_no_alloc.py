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


@pytest.mark.parametrize("prec", ["f64", "f32", "f16q"])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 4, 2, 10)])
def test_static_scratch_plaquette_matches(dims, prec):
    lat = Lattice(dims, 2.4, seed=3, start="hot", prec=prec)
    lat.sweep(2)
    for _ in range(2):                       # two calls in a row share the fixed scratch
        ref = lat.plaquette()
        got = static_plaquette(lat)
        np.testing.assert_allclose(got, ref, atol=MTOL[prec], rtol=0)
        assert np.abs(got - static_plaquette(lat)).max() == 0.0
        lat.sweep(1)                         # a different configuration for the next call
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
