"""ctypes view of the plain FP64 CPU oracle (su2_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the package smoke check
and the CPU-baseline leg of the benchmark; the product path never imports it.
Arrays are numpy float64 in the canonical layout U[s, mu, c] with
s = x0 + N0*(x1 + N1*(x2 + N2*x3)); see su2_oracle.h for the conventions and
the paper passages each function follows.
"""
import contextlib
import ctypes as C

import numpy as np

from . import build as _build

_lib = None

KP = 0
CREUTZ = 1


class Chain(C.Structure):
    _fields_ = [("beta", C.c_double), ("seed", C.c_uint64), ("lattice_id", C.c_uint32),
                ("max_tries", C.c_int), ("sampler", C.c_int), ("u23", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("updates", C.c_uint64), ("trials", C.c_uint64), ("capped", C.c_uint64),
                ("haar", C.c_uint64)]


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_up = C.POINTER(C.c_uint32)


def _load(path):
    L = C.CDLL(path)
    sig = {
        "oracle_threads": (C.c_int, []),
        "oracle_philox4x32_10": (None, [_up, _up, _up]),
        "oracle_u01": (C.c_double, [C.c_uint32, C.c_int]),
        "oracle_draw": (None, [C.POINTER(Chain), C.c_long, C.c_int, C.c_uint32, C.c_uint32, _dp]),
        "oracle_qmul": (None, [_dp, _dp, _dp]),
        "oracle_qdag": (None, [_dp, _dp]),
        "oracle_volume": (C.c_long, [C.c_int, _ip]),
        "oracle_shift": (C.c_long, [C.c_int, _ip, C.c_long, C.c_int, C.c_int]),
        "oracle_init_cold": (None, [C.c_int, _ip, _dp]),
        "oracle_init_hot": (None, [C.c_int, _ip, C.POINTER(Chain), _dp]),
        "oracle_hot_link": (None, [C.POINTER(Chain), C.c_long, C.c_int, _dp]),
        "oracle_staple": (None, [C.c_int, _ip, _dp, C.c_long, C.c_int, _dp]),
        "oracle_sample_a0": (C.c_int, [C.POINTER(Chain), C.c_double, C.c_long, C.c_int,
                                       C.c_uint32, _dp, _dp]),
        "oracle_heatbath_link": (C.c_int, [C.POINTER(Chain), C.c_long, C.c_int, C.c_uint32,
                                           _dp, _dp, _dp, _dp]),
        "oracle_substep": (None, [C.c_int, _ip, _dp, C.POINTER(Chain), C.c_uint32, C.c_int,
                                  C.c_int, C.POINTER(Stats), _dp]),
        "oracle_sweep": (None, [C.c_int, _ip, _dp, C.POINTER(Chain), C.c_uint32,
                                C.POINTER(Stats)]),
        "oracle_overrelax_substep": (None, [C.c_int, _ip, _dp, C.c_int, C.c_int]),
        "oracle_plaquette": (None, [C.c_int, _ip, _dp, _dp]),
        "oracle_polyakov": (C.c_double, [C.c_int, _ip, _dp]),
        "oracle_wilson_loops": (None, [C.c_int, _ip, _dp, C.c_int, C.c_int, _dp]),
        "oracle_ape_step": (None, [C.c_int, _ip, _dp, _dp, C.c_double]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


def lib():
    global _lib
    if _lib is None:
        _lib = _load(_build.build())
    return _lib


def threads():
    """Threads the bound build's substep loop uses (1 for the serial build)."""
    return lib().oracle_threads()


@contextlib.contextmanager
def parallel():
    """Bind this module to the OpenMP build of the same source (all host
    cores share the sites of each substep; results are those of the serial
    build) for the duration of the block."""
    with using_library(_build.build(omp=True)):
        yield


@contextlib.contextmanager
def using_library(path):
    """Temporarily bind this module to another build of su2_oracle.c (the
    tests use it to show that a planted mistake fails the pins)."""
    global _lib
    saved = _lib
    _lib = _load(path)
    try:
        yield
    finally:
        _lib = saved


def _d(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _dims(dims):
    arr = (C.c_int * len(dims))(*dims)
    return len(dims), arr


def chain(beta, seed=1, lattice_id=0, max_tries=64, sampler=KP, u23=0):
    return Chain(float(beta), int(seed), int(lattice_id), int(max_tries), int(sampler), int(u23))


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (C.c_uint32 * 4)()
    lib().oracle_philox4x32_10(c, k, o)
    return [o[i] for i in range(4)]


def u01(x, u23=0):
    return lib().oracle_u01(int(x) & 0xFFFFFFFF, int(u23))


def qmul(a, b):
    a = np.ascontiguousarray(a, np.float64)
    b = np.ascontiguousarray(b, np.float64)
    o = np.empty(4)
    lib().oracle_qmul(_d(a), _d(b), _d(o))
    return o


def qdag(a):
    a = np.ascontiguousarray(a, np.float64)
    o = np.empty(4)
    lib().oracle_qdag(_d(a), _d(o))
    return o


def volume(dims):
    return int(np.prod(dims))


def empty_field(dims):
    return np.empty((volume(dims), len(dims), 4), np.float64)


def init_cold(dims):
    U = empty_field(dims)
    nd, d = _dims(dims)
    lib().oracle_init_cold(nd, d, _d(U))
    return U


def init_hot(dims, ch):
    U = empty_field(dims)
    nd, d = _dims(dims)
    lib().oracle_init_hot(nd, d, C.byref(ch), _d(U))
    return U


def hot_link(ch, s, mu):
    o = np.empty(4)
    lib().oracle_hot_link(C.byref(ch), int(s), int(mu), _d(o))
    return o


def staple(dims, U, s, mu):
    nd, d = _dims(dims)
    o = np.empty(4)
    lib().oracle_staple(nd, d, _d(U), int(s), int(mu), _d(o))
    return o


def sample_a0(ch, alpha, s, mu, sweep):
    a0 = C.c_double(np.nan)
    m = C.c_double()
    n = lib().oracle_sample_a0(C.byref(ch), float(alpha), int(s), int(mu), int(sweep),
                               C.byref(a0), C.byref(m))
    return n, a0.value, m.value


def heatbath_link(ch, s, mu, sweep, sigma, old):
    sigma = np.ascontiguousarray(sigma, np.float64)
    old = np.ascontiguousarray(old, np.float64)
    o = np.empty(4)
    m = C.c_double()
    n = lib().oracle_heatbath_link(C.byref(ch), int(s), int(mu), int(sweep), _d(sigma), _d(old),
                                   _d(o), C.byref(m))
    return n, o, m.value


def substep(dims, U, ch, sweep, mu, parity, margins=False):
    nd, d = _dims(dims)
    st = Stats()
    marg = np.full((volume(dims), nd), np.inf) if margins else None
    lib().oracle_substep(nd, d, _d(U), C.byref(ch), int(sweep), int(mu), int(parity),
                         C.byref(st), _d(marg) if margins else None)
    return (st, marg) if margins else st


def sweep(dims, U, ch, sweep_index):
    nd, d = _dims(dims)
    st = Stats()
    lib().oracle_sweep(nd, d, _d(U), C.byref(ch), int(sweep_index), C.byref(st))
    return st


def overrelax_substep(dims, U, mu, parity):
    nd, d = _dims(dims)
    lib().oracle_overrelax_substep(nd, d, _d(U), int(mu), int(parity))


def plaquette(dims, U):
    nd, d = _dims(dims)
    o = np.empty(3)
    lib().oracle_plaquette(nd, d, _d(U), _d(o))
    return o


def polyakov(dims, U):
    nd, d = _dims(dims)
    return lib().oracle_polyakov(nd, d, _d(U))


def wilson_loops(dims, U, rmax, tmax):
    nd, d = _dims(dims)
    o = np.empty((rmax, tmax))
    lib().oracle_wilson_loops(nd, d, _d(U), int(rmax), int(tmax), _d(o))
    return o


def ape_step(dims, U, alpha):
    nd, d = _dims(dims)
    O = np.empty_like(U)
    lib().oracle_ape_step(nd, d, _d(U), _d(O), float(alpha))
    return O


def ape_smear(dims, U, alpha, n):
    for _ in range(n):
        U = ape_step(dims, U, alpha)
    return U
