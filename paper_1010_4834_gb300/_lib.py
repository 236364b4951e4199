"""ctypes declarations of libsu2 (include/su2.h).  Argument marshalling only.

The shared library is built by paper_1010_4834_gb300.build (nvcc, sm_103a) into
paper_1010_4834_gb300/_build/libsu2.so.  There is no CPU fallback: if the
library is missing, loading raises.
"""
import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsu2.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "su2.h")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ESTATE = 0, 1, 2, 3, 4, 5
COLD, HOT = 0, 1
F64, F32, F16Q = 0, 1, 2
SAMPLER_KP, SAMPLER_CREUTZ = 0, 1
SCHED_AUTO, SCHED_SUBSTEP, SCHED_PAIR = 0, 1, 2
SCHEDULE = {"auto": SCHED_AUTO, "substep": SCHED_SUBSTEP, "pair": SCHED_PAIR}

PREC = {"f64": F64, "f32": F32, "f16q": F16Q, F64: F64, F32: F32, F16Q: F16Q}
START = {"cold": COLD, "hot": HOT, COLD: COLD, HOT: HOT}
STATUS = {EINVAL: "SU2_EINVAL", ENOMEM: "SU2_ENOMEM", ECUDA: "SU2_ECUDA",
          ETIMEOUT: "SU2_ETIMEOUT", ESTATE: "SU2_ESTATE"}


class SU2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, str(code)), msg))
        self.code = code


_vp = C.c_void_p
_pp = C.POINTER(C.c_void_p)
_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)
_i, _u32, _u64, _d, _sz, _s = C.c_int, C.c_uint32, C.c_uint64, C.c_double, C.c_size_t, C.c_char_p

SIGNATURES = {
    "su2_last_error": (_s, []),
    "su2_version": (_s, []),
    "su2_required_bytes": (_i, [_ip, _i, C.POINTER(_sz)]),
    "su2_init": (_i, [_pp, _ip, _d, _u64, _i, _i, _vp]),
    "su2_init_external": (_i, [_pp, _ip, _d, _u64, _i, _i, _vp, _sz, _vp]),
    "su2_destroy": (_i, [_vp]),
    "su2_set_stream": (_i, [_vp, _vp]),
    "su2_set_options": (_i, [_vp, _i, _i]),
    "su2_set_beta": (_i, [_vp, _d]),
    "su2_set_schedule": (_i, [_vp, _i]),
    "su2_set_overrelax": (_i, [_vp, _i]),
    "su2_heatbath_sweep": (_i, [_vp, _i]),
    "su2_heatbath_substep": (_i, [_vp, _i, _i, _u32]),
    "su2_heatbath_pair": (_i, [_vp, _i, _u32]),
    "su2_restart": (_i, [_vp, _i]),
    "su2_sweep_measure": (_i, [_vp, _i, _dp]),
    "su2_layout_compare": (_i, [_vp, _i, _dp, C.POINTER(_u64)]),
    "su2_kernel_launches": (_i, [C.POINTER(_u64)]),
    "su2_probe_fma": (_i, [_i, _i, _dp]),
    "su2_overrelax_sweep": (_i, [_vp, _i]),
    "su2_plaquette": (_i, [_vp, _dp]),
    "su2_plaquette_static": (_i, [_vp, _ip, _i, _dp, _vp]),
    "su2_polyakov": (_i, [_vp, _dp]),
    "su2_set_site_offset": (_i, [_vp, _u32]),
    "su2_plaquette_slices": (_i, [_vp, _i, _i, _dp]),
    "su2_time_lines": (_i, [_vp, _i, _i, _dp]),
    "su2_ape_smear": (_i, [_vp, _d, _i]),
    "su2_wilson_loops": (_i, [_vp, _i, _i, _i, _dp]),
    "su2_get_links": (_i, [_vp, _dp]),
    "su2_get_sites": (_i, [_vp, C.c_int64, C.c_int64, _dp]),
    "su2_set_links": (_i, [_vp, _dp]),
    "su2_sweep_count": (_i, [_vp, C.POINTER(_u64)]),
    "su2_set_sweep_count": (_i, [_vp, _u64]),
    "su2_save": (_i, [_vp, _s]),
    "su2_load": (_i, [_pp, _s, _i, _vp]),
    "su2_batch_init": (_i, [_pp, _i, _ip, _dp, _u64, _i, _i, _vp]),
    "su2_batch_destroy": (_i, [_vp]),
    "su2_batch_set_options": (_i, [_vp, _i, _i]),
    "su2_batch_set_overrelax": (_i, [_vp, _i]),
    "su2_batch_sweep": (_i, [_vp, _i]),
    "su2_batch_sweep_measure": (_i, [_vp, _i, _dp]),
    "su2_batch_set_groups": (_i, [_vp, _i]),
    "su2_batch_groups": (_i, [_vp, _ip]),
    "su2_batch_set_block_size": (_i, [_vp, _i]),
    "su2_batch_block_size": (_i, [_vp, _ip]),
    "su2_batch_tune": (_i, [_vp, _i, _ip]),
    "su2_batch_plaquette": (_i, [_vp, _dp]),
    "su2_batch_polyakov": (_i, [_vp, _dp]),
    "su2_batch_get_links": (_i, [_vp, _i, _dp]),
    "su2_batch_set_links": (_i, [_vp, _i, _dp]),
}

_lib = None


def header_functions():
    """Names of the functions include/su2.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(su2_\w+)\s*\(", text)))


def load(path=None):
    """Load libsu2.so and declare every signature; raise if it is not built."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libsu2.so is not built (%s); run paper_1010_4834_gb300.build.build() "
                           "or __graft_entry__.build() first" % p)
    L = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = L
    return L


def check(rc):
    if rc != OK:
        raise SU2Error(rc, load().su2_last_error().decode())
    return rc


def dims_arg(dims):
    if len(dims) != 4:
        raise ValueError("dims must have 4 extents")
    return (C.c_int * 4)(*[int(d) for d in dims])
