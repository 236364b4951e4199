"""Python view of libsu2: `Lattice` and `Batch`.

Thin marshalling over the C ABI of include/su2.h.  Every step of the Monte
Carlo runs in the library's CUDA kernels; PyTorch only supplies device memory
(the link store lives in a torch uint8 tensor handed to su2_init_external) and
the CUDA stream (torch's current stream unless one is given).
"""
import ctypes as C

import numpy as np

from . import _lib
from ._lib import check, dims_arg


_CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy: the implicit default stream


def _stream_ptr(stream):
    """torch's stream as a cudaStream_t.  torch's default stream has handle 0,
    which the C ABI reads as "create a private stream"; pass the legacy
    default stream's handle instead so the work stays ordered with torch."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    h = int(s.cuda_stream)
    return C.c_void_p(h if h != 0 else _CUDA_STREAM_LEGACY)


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def kernel_launches():
    """Kernels libsu2 has launched in this process."""
    n = C.c_uint64()
    check(_lib.load().su2_kernel_launches(C.byref(n)))
    return n.value


def probe_fma(prec="f64", iters=1 << 14):
    """This device's FMA throughput in flop/s (su2_probe_fma)."""
    v = C.c_double()
    check(_lib.load().su2_probe_fma(_lib.PREC[prec], int(iters), C.byref(v)))
    return v.value


def required_bytes(dims, prec):
    """Device bytes a lattice of these extents and precision needs."""
    n = C.c_size_t()
    check(_lib.load().su2_required_bytes(dims_arg(tuple(int(d) for d in dims)), _lib.PREC[prec], C.byref(n)))
    return n.value


class Lattice:
    """One SU(2) lattice with links on the GPU (see include/su2.h).

    dims: (N0, N1, N2, N3), each even >= 2.  start: "cold" | "hot".
    prec: "f64" | "f32" | "f16q".  Device memory comes from torch unless
    torch_memory=False (the library then calls cudaMalloc itself).
    """

    def __init__(self, dims, beta, seed=1, start="cold", prec="f32", stream=None,
                 torch_memory=True, _handle=None):
        import torch
        L = _lib.load()
        self.dims = tuple(int(d) for d in dims)
        self.prec = _lib.PREC[prec]
        self._buf = None
        self._stream = stream
        h = C.c_void_p()
        if _handle is not None:
            h = _handle
        elif torch_memory:
            nbytes = C.c_size_t()
            check(L.su2_required_bytes(dims_arg(self.dims), self.prec, C.byref(nbytes)))
            self._buf = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
            check(L.su2_init_external(C.byref(h), dims_arg(self.dims), float(beta), int(seed),
                                      _lib.START[start], self.prec, C.c_void_p(self._buf.data_ptr()),
                                      nbytes.value, _stream_ptr(stream)))
        else:
            check(L.su2_init(C.byref(h), dims_arg(self.dims), float(beta), int(seed),
                             _lib.START[start], self.prec, _stream_ptr(stream)))
        self._h = h

    @property
    def volume(self):
        return int(np.prod(self.dims))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            check(_lib.load().su2_destroy(self._h))
            self._h = C.c_void_p()
        self._buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- chain ------------------------------------------------------------
    def set_options(self, max_tries=64, sampler="kp"):
        s = {"kp": _lib.SAMPLER_KP, "creutz": _lib.SAMPLER_CREUTZ}.get(sampler, sampler)
        check(_lib.load().su2_set_options(self._h, int(max_tries), int(s)))

    def set_beta(self, beta):
        check(_lib.load().su2_set_beta(self._h, float(beta)))

    def set_schedule(self, schedule="auto"):
        """Heat-bath sweep launches: "auto", "substep" or "pair" (su2_set_schedule)."""
        check(_lib.load().su2_set_schedule(self._h, _lib.SCHEDULE.get(schedule, schedule)))

    def set_overrelax(self, n):
        """n over-relaxation sweeps before every heat-bath sweep (su2_set_overrelax)."""
        check(_lib.load().su2_set_overrelax(self._h, int(n)))

    def sweep(self, n=1):
        check(_lib.load().su2_heatbath_sweep(self._h, int(n)))

    def restart(self, start="hot"):
        check(_lib.load().su2_restart(self._h, _lib.START[start]))

    def sweep_measure(self, n, out=None):
        """n x (sweep, plaquette, Polyakov); returns an (n, 4) array:
        plaquette all / spatial / space-time, Polyakov loop."""
        if out is None:
            out = np.empty((n, 4))
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.size >= 4 * n
        check(_lib.load().su2_sweep_measure(self._h, int(n), _dptr(out)))
        return out

    def layout_compare(self, sweeps):
        """Section 5.1's layout comparison on this GPU (FP32): ms of `sweeps`
        sweeps with the library's kernels, with a plain kernel on the
        library's layout and on a site-major single array, and the number of
        links in which the latter two results differ from the first."""
        ms = np.empty(3)
        n = C.c_uint64()
        check(_lib.load().su2_layout_compare(self._h, int(sweeps), _dptr(ms), C.byref(n)))
        return ms, n.value

    def substep(self, mu, parity, sweep_index):
        check(_lib.load().su2_heatbath_substep(self._h, int(mu), int(parity), int(sweep_index)))

    def pair(self, mu, sweep_index):
        """Both parities of direction mu in one fused launch (su2_heatbath_pair)."""
        check(_lib.load().su2_heatbath_pair(self._h, int(mu), int(sweep_index)))

    def overrelax(self, n=1):
        check(_lib.load().su2_overrelax_sweep(self._h, int(n)))

    @property
    def sweep_count(self):
        n = C.c_uint64()
        check(_lib.load().su2_sweep_count(self._h, C.byref(n)))
        return n.value

    @sweep_count.setter
    def sweep_count(self, n):
        check(_lib.load().su2_set_sweep_count(self._h, int(n)))

    # -- measurements -----------------------------------------------------
    def plaquette(self):
        out = np.empty(3)
        check(_lib.load().su2_plaquette(self._h, _dptr(out)))
        return out

    def set_site_offset(self, site0):
        """Philox site word offset of this lattice (su2_set_site_offset)."""
        check(_lib.load().su2_set_site_offset(self._h, int(site0) & 0xFFFFFFFF))

    def plaquette_slices(self, t_first, t_count):
        """Plaquette means over base sites in time slices [t_first, t_first + t_count)."""
        out = np.empty(3)
        check(_lib.load().su2_plaquette_slices(self._h, int(t_first), int(t_count), _dptr(out)))
        return out

    def time_lines(self, t_first, t_count):
        """Ordered products of the time links of slices [t_first, t_first + t_count)
        per spatial site: shape (N0 N1 N2, 4)."""
        out = np.empty((self.volume // self.dims[3], 4))
        check(_lib.load().su2_time_lines(self._h, int(t_first), int(t_count), _dptr(out)))
        return out

    def polyakov(self):
        v = C.c_double()
        check(_lib.load().su2_polyakov(self._h, C.byref(v)))
        return v.value

    def ape_smear(self, alpha, n):
        check(_lib.load().su2_ape_smear(self._h, float(alpha), int(n)))

    def wilson_loops(self, rmax, tmax, smeared=False):
        out = np.empty((rmax, tmax))
        check(_lib.load().su2_wilson_loops(self._h, int(rmax), int(tmax), int(bool(smeared)), _dptr(out)))
        return out

    # -- links ------------------------------------------------------------
    def get_links(self, out=None):
        """Canonical FP64 links, shape (V, 4, 4) = (site, direction, component)."""
        if out is None:
            out = np.empty((self.volume, 4, 4))
        assert out.dtype == np.float64 and out.flags.c_contiguous and out.size == self.volume * 16
        check(_lib.load().su2_get_links(self._h, _dptr(out)))
        return out

    def get_sites(self, first, count):
        """Canonical FP64 links of sites [first, first + count): shape (count, 4, 4)."""
        out = np.empty((int(count), 4, 4))
        check(_lib.load().su2_get_sites(self._h, int(first), int(count), _dptr(out)))
        return out

    def set_links(self, U):
        """Canonical FP64 links (V, 4, 4) from a numpy array, or from a
        contiguous float64 CUDA tensor on the lattice's device, which must be
        ready on the lattice's stream (the library reads it there)."""
        if hasattr(U, "is_cuda") and U.is_cuda:
            import torch
            assert U.dtype == torch.float64 and U.is_contiguous() and U.numel() == self.volume * 16
            check(_lib.load().su2_set_links(self._h, C.cast(C.c_void_p(U.data_ptr()), C.POINTER(C.c_double))))
            return
        U = np.ascontiguousarray(U, np.float64)
        assert U.size == self.volume * 16
        check(_lib.load().su2_set_links(self._h, _dptr(U)))

    def save(self, path):
        check(_lib.load().su2_save(self._h, str(path).encode()))

    @classmethod
    def load(cls, path, prec=-1, stream=None):
        h = C.c_void_p()
        p = _lib.PREC[prec] if prec != -1 else -1
        check(_lib.load().su2_load(C.byref(h), str(path).encode(), int(p), _stream_ptr(stream)))
        # dims/prec from the file header: read back via a small parse
        import struct
        with open(path, "rb") as f:
            head = f.read(8 + 4 + 16 + 4)
        dims = struct.unpack("<4i", head[12:28])
        prec_saved = struct.unpack("<i", head[28:32])[0]
        obj = cls.__new__(cls)
        obj.dims = tuple(dims)
        obj.prec = prec_saved if p == -1 else p
        obj._buf = None
        obj._stream = stream
        obj._h = h
        return obj


class Batch:
    """Many independent lattices swept together (su2_batch_* in include/su2.h)."""

    def __init__(self, dims_list, betas, seed=1, start="hot", prec="f32", stream=None):
        L = _lib.load()
        self.prec_name = {v: k for k, v in _lib.PREC.items() if isinstance(k, str)}[_lib.PREC[prec]]
        self.dims = [tuple(int(d) for d in dd) for dd in dims_list]
        n = len(self.dims)
        flat = (C.c_int * (4 * n))(*[d for dd in self.dims for d in dd])
        b = np.ascontiguousarray(betas, np.float64)
        assert len(b) == n
        h = C.c_void_p()
        check(L.su2_batch_init(C.byref(h), n, flat, _dptr(b), int(seed), _lib.START[start],
                               _lib.PREC[prec], _stream_ptr(stream)))
        self._h = h
        self.n = n

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            check(_lib.load().su2_batch_destroy(self._h))
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_options(self, max_tries=64, sampler="kp"):
        s = {"kp": _lib.SAMPLER_KP, "creutz": _lib.SAMPLER_CREUTZ}.get(sampler, sampler)
        check(_lib.load().su2_batch_set_options(self._h, int(max_tries), int(s)))

    def set_overrelax(self, n):
        """n over-relaxation sweeps before each heat-bath sweep (su2_batch_set_overrelax)."""
        check(_lib.load().su2_batch_set_overrelax(self._h, int(n)))

    def sweep(self, n=1):
        check(_lib.load().su2_batch_sweep(self._h, int(n)))

    def sweep_measure(self, n):
        """n sweeps, each followed by every lattice's plaquette (all,
        spatial, space-time) and Polyakov loop: an (n, lattices, 4) array
        (su2_batch_sweep_measure)."""
        out = np.empty((int(n), self.n, 4))
        check(_lib.load().su2_batch_sweep_measure(self._h, int(n), _dptr(out)))
        return out

    @property
    def groups(self):
        g = C.c_int()
        check(_lib.load().su2_batch_groups(self._h, C.byref(g)))
        return g.value

    @groups.setter
    def groups(self, g):
        check(_lib.load().su2_batch_set_groups(self._h, int(g)))

    @property
    def block_size(self):
        t = C.c_int()
        check(_lib.load().su2_batch_block_size(self._h, C.byref(t)))
        return t.value

    @block_size.setter
    def block_size(self, threads):
        check(_lib.load().su2_batch_set_block_size(self._h, int(threads)))

    def tune(self, sweeps=4, cache=False):
        """Pick the fastest (block size, group count) on a scratch copy;
        returns the group count (block_size gives the other).  With
        cache (True, or a file path) a group count recorded for this GPU,
        precision and set of shapes is applied without timing, and a new
        result is recorded (paper_1010_4834_gb300.tuning)."""
        from . import tuning
        path = cache if isinstance(cache, str) else None
        k = None
        if cache:
            import torch
            k = tuning.key(torch.cuda.get_device_name(), self.prec_name, self.dims)
            hit = tuning.lookup(k, path)
            if hit is not None:
                self.block_size = int(hit.get("block_size", 256))
                self.groups = int(hit["groups"])
                return self.groups
        g = C.c_int()
        check(_lib.load().su2_batch_tune(self._h, int(sweeps), C.byref(g)))
        if k is not None:
            tuning.store(k, {"groups": g.value, "block_size": self.block_size, "sweeps_timed": int(sweeps)}, path)
        return g.value

    def plaquette(self):
        out = np.empty((self.n, 3))
        check(_lib.load().su2_batch_plaquette(self._h, _dptr(out)))
        return out

    def set_site_offset(self, site0):
        """Philox site word offset of this lattice (su2_set_site_offset)."""
        check(_lib.load().su2_set_site_offset(self._h, int(site0) & 0xFFFFFFFF))

    def plaquette_slices(self, t_first, t_count):
        """Plaquette means over base sites in time slices [t_first, t_first + t_count)."""
        out = np.empty(3)
        check(_lib.load().su2_plaquette_slices(self._h, int(t_first), int(t_count), _dptr(out)))
        return out

    def time_lines(self, t_first, t_count):
        """Ordered products of the time links of slices [t_first, t_first + t_count)
        per spatial site: shape (N0 N1 N2, 4)."""
        out = np.empty((self.volume // self.dims[3], 4))
        check(_lib.load().su2_time_lines(self._h, int(t_first), int(t_count), _dptr(out)))
        return out

    def polyakov(self):
        out = np.empty(self.n)
        check(_lib.load().su2_batch_polyakov(self._h, _dptr(out)))
        return out

    def get_links(self, i):
        V = int(np.prod(self.dims[i]))
        out = np.empty((V, 4, 4))
        check(_lib.load().su2_batch_get_links(self._h, int(i), _dptr(out)))
        return out

    def set_links(self, i, U):
        U = np.ascontiguousarray(U, np.float64)
        check(_lib.load().su2_batch_set_links(self._h, int(i), _dptr(U)))
