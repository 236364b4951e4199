"""The C-ABI library loads on any host and exports every function include/su2.h declares.

No compute call is made here (no GPU needed); su2_required_bytes and
argument validation touch no device.
"""
import ctypes as C

import pytest

from paper_1010_4834_gb300 import _lib


@pytest.fixture(scope="module")
def lib():
    from paper_1010_4834_gb300 import build
    build.build()
    return _lib.load()


def test_every_declared_function_is_exported(lib):
    names = _lib.header_functions()
    assert len(names) >= 30
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each
    assert sorted(_lib.SIGNATURES) == names


def test_required_bytes_and_validation(lib):
    n = C.c_size_t()
    assert lib.su2_required_bytes(_lib.dims_arg([8, 8, 8, 8]), _lib.F32, C.byref(n)) == _lib.OK
    V = 8 ** 4
    assert n.value >= 10 * V * 16          # links + two spatial APE buffers
    m = C.c_size_t()
    lib.su2_required_bytes(_lib.dims_arg([8, 8, 8, 8]), _lib.F64, C.byref(m))
    assert m.value > n.value
    for bad in ([7, 8, 8, 8], [8, 0, 8, 8], [8, 8, -2, 8]):
        assert lib.su2_required_bytes(_lib.dims_arg(bad), _lib.F32, C.byref(n)) == _lib.EINVAL
        assert b"even" in lib.su2_last_error()
    assert lib.su2_required_bytes(_lib.dims_arg([8, 8, 8, 8]), 7, C.byref(n)) == _lib.EINVAL
    h = C.c_void_p()
    assert lib.su2_init(C.byref(h), _lib.dims_arg([8, 8, 8, 9]), 2.0, 1, 0, 1, None) == _lib.EINVAL
    assert lib.su2_init(C.byref(h), _lib.dims_arg([8, 8, 8, 8]), -1.0, 1, 0, 1, None) == _lib.EINVAL
    assert lib.su2_init(C.byref(h), _lib.dims_arg([8, 8, 8, 8]), 2.0, 1, 5, 1, None) == _lib.EINVAL
    assert lib.su2_destroy(None) == _lib.OK
    assert lib.su2_heatbath_sweep(None, 1) == _lib.EINVAL
    assert lib.su2_version().startswith(b"su2-gb300")
