"""Domain decomposition of one lattice into time slabs, one per GPU
(Section 4: the paper's multi-GPU code splits the lattice along the time
direction, each GPU holding its own slices plus a ghost slice on each side,
and exchanges the border slices before each update).

Rank r of G owns global time slices [t0, t0 + n), t0 = r n, n = Nt / G, and
holds them as a lattice of its own with extents (N0, N1, N2, n + 2): local
slices 1..n are its own, local slices 0 and n + 1 copy the neighbouring
slabs' boundary slices (global t0 - 1 and t0 + n, periodic).  n is even, so
every local slice 0 lies an odd number of slices before global slice 0 and a
local site's parity is its global parity xor 1 on every slab.  The slab's
Philox site word is shifted by (t0 - 1) N0 N1 N2 (su2_set_site_offset), so
its draws are those of the whole lattice.

A heat-bath substep (mu, p) of the whole lattice is, on every slab, the
substep (mu, p xor 1) of its local lattice followed by the exchange of the
updated class's boundary slices: local slice 1 goes to the lower
neighbour's ghost n + 1 and local slice n to the upper neighbour's ghost 0.
The local substep also updates the ghost slices' links, from wrapped-around
neighbours; those values are never used, since the exchange overwrites
them.  Only the class that changed moves, so every ghost is current before
each substep, and the slabs' own links are those of the undivided lattice.
A measured sweep adds one all-reduce (the plaquettes based on each slab's own
slices) and one all-gather of partial time lines, whose product in time
order is the Polyakov loop (Eqs. 14-15).

The module holds only the decomposition and the exchange.  The arithmetic
is a slab store's: SlabLattice runs it in the library's kernels; the tests
define a store on the CPU oracle.  Communication is a comm object: TorchComm
over a torch.distributed process group (gloo for host buffers, NCCL for
device buffers on several GPUs), or ThreadWorld, which runs the ranks as host
threads of one process and moves slices through queues.
"""
import queue
import threading

import numpy as np


class SlabGeometry:
    """Rank `rank` of `world` time slabs of a lattice of extents `dims`."""

    def __init__(self, dims, world, rank):
        dims = tuple(int(d) for d in dims)
        nt = dims[3]
        if world < 1 or nt % world or (nt // world) % 2 or nt // world < 2:
            raise ValueError("Nt = %d must split into %d slabs of an even number (>= 2) of slices" % (nt, world))
        self.dims, self.world, self.rank = dims, world, rank
        self.n = nt // world
        self.t0 = rank * self.n
        self.local_dims = dims[:3] + (self.n + 2,)
        self.nsig = dims[0] * dims[1] * dims[2]
        self.volume = self.nsig * nt
        # the Philox site word of local site s is s + site0 (mod 2^32)
        self.site0 = ((self.t0 - 1) * self.nsig) % (1 << 32)
        self.lower = (rank - 1) % world
        self.upper = (rank + 1) % world

    @staticmethod
    def local_parity(p):
        """The local class of global parity p (local slice 0 is global t0 - 1, t0 even)."""
        return p ^ 1

    def global_slice(self, t_local):
        return (self.t0 - 1 + t_local) % self.dims[3]

    def local_config(self, U):
        """The slab's local configuration (ghosts included) cut from a whole
        canonical configuration U[s, mu, c]."""
        U = np.asarray(U)
        rows = [U[self.global_slice(t) * self.nsig:(self.global_slice(t) + 1) * self.nsig]
                for t in range(self.n + 2)]
        return np.concatenate(rows, axis=0)

    def own_part(self, U_local):
        """The slab's own slices (1..n) of a local canonical configuration."""
        return np.asarray(U_local)[self.nsig:(self.n + 1) * self.nsig]


# ---------------------------------------------------------------------------
# the distributed algorithm, per rank
# ---------------------------------------------------------------------------
def exchange_class(store, comm, geom, mu, p_local):
    """Refresh the neighbours' ghosts of class (mu, p_local) after it changed."""
    to_lower = store.get_slice(1, mu, p_local)
    to_upper = store.get_slice(geom.n, mu, p_local)
    from_lower, from_upper = comm.exchange(to_lower, to_upper)
    store.set_slice(0, mu, p_local, from_lower)
    store.set_slice(geom.n + 1, mu, p_local, from_upper)


def fill_ghosts(store, comm, geom):
    """Make every ghost class current (after the slabs' links were set)."""
    for mu in range(4):
        for p in range(2):
            exchange_class(store, comm, geom, mu, p)


def sweep(store, comm, geom, sweep_index):
    """One heat-bath sweep of the whole lattice (direction outer, parity
    inner, as the undivided lattice runs it) with Philox sweep index
    `sweep_index`."""
    for mu in range(4):
        for p in range(2):
            pl = geom.local_parity(p)
            store.substep(mu, pl, sweep_index)
            exchange_class(store, comm, geom, mu, pl)


def plaquette(store, comm, geom):
    """{all, spatial, space-time} plaquette means of the whole lattice."""
    m = np.asarray(store.plaquette_slices(1, geom.n), float)
    # means over 3 nsig n plaquettes per part -> sums -> whole-lattice means
    sums = np.array([2 * m[0], m[1], m[2]]) * 3 * geom.nsig * geom.n
    tot = comm.allreduce_sum(sums)
    n3 = 3.0 * geom.volume
    return np.array([tot[0] / (2 * n3), tot[1] / n3, tot[2] / n3])


def qmul_lines(a, b):
    """Product a b of quaternion arrays (..., 4) (Section 2, Eq. 1 algebra)."""
    w = a[..., 0] * b[..., 0] - a[..., 1] * b[..., 1] - a[..., 2] * b[..., 2] - a[..., 3] * b[..., 3]
    x = a[..., 0] * b[..., 1] + a[..., 1] * b[..., 0] - a[..., 2] * b[..., 3] + a[..., 3] * b[..., 2]
    y = a[..., 0] * b[..., 2] + a[..., 2] * b[..., 0] - a[..., 3] * b[..., 1] + a[..., 1] * b[..., 3]
    z = a[..., 0] * b[..., 3] + a[..., 3] * b[..., 0] - a[..., 1] * b[..., 2] + a[..., 2] * b[..., 1]
    return np.stack([w, x, y, z], axis=-1)


def polyakov(store, comm, geom):
    """Signed Polyakov loop of the whole lattice: each slab's time lines over
    its own slices, multiplied in rank (= time) order."""
    lines = comm.allgather(np.asarray(store.time_lines(1, geom.n), float))
    pr = lines[0]
    for l in lines[1:]:
        pr = qmul_lines(pr, l)
    return float(pr[:, 0].mean())


# ---------------------------------------------------------------------------
# communication
# ---------------------------------------------------------------------------
class TorchComm:
    """Exchange and reductions over a torch.distributed process group.
    Slices travel as torch tensors (host tensors with gloo, device tensors
    with NCCL); reductions as float64 tensors on `device`."""

    def __init__(self, group=None, device="cpu"):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.device = device

    def exchange(self, to_lower, to_upper):
        import torch
        dist = self.dist
        lower, upper = (self.rank - 1) % self.world, (self.rank + 1) % self.world
        to_lower, to_upper = torch.as_tensor(to_lower), torch.as_tensor(to_upper)
        if self.world == 1:
            return to_upper.clone(), to_lower.clone()
        from_lower, from_upper = torch.empty_like(to_upper), torch.empty_like(to_lower)
        # sends and receives in matching order (NCCL pairs them by order, with
        # two ranks both go to the same peer): the upper neighbour's lower
        # ghost receives this rank's last slice, the lower neighbour's upper
        # ghost its first; tags say the same for backends that use them
        ops = [dist.P2POp(dist.isend, to_upper, upper, self.group, tag=1),
               dist.P2POp(dist.isend, to_lower, lower, self.group, tag=0),
               dist.P2POp(dist.irecv, from_lower, lower, self.group, tag=1),
               dist.P2POp(dist.irecv, from_upper, upper, self.group, tag=0)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        return from_lower, from_upper

    def allreduce_sum(self, x):
        import torch
        t = torch.as_tensor(np.asarray(x, np.float64), device=self.device).clone()
        self.dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()

    def allgather(self, x):
        import torch
        t = torch.as_tensor(np.asarray(x, np.float64), device=self.device).contiguous()
        out = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t, group=self.group)
        return [o.cpu().numpy() for o in out]


class ThreadWorld:
    """G ranks as host threads of one process: run(fn) calls fn(rank, comm)
    on every rank concurrently and returns the results in rank order.
    Slices are handed over as they are (the stores copy them in)."""

    def __init__(self, world):
        self.world = world
        self.q = {(a, b): queue.Queue() for a in range(world) for b in range(world)}
        self.barrier = threading.Barrier(world)
        self.slots = [None] * world

    class _Comm:
        def __init__(self, w, rank):
            self.w, self.rank, self.world = w, rank, w.world

        def exchange(self, to_lower, to_upper):
            # a rank's lower ghost is its lower neighbour's "to_upper" slice,
            # its upper ghost the upper neighbour's "to_lower" slice (with one
            # or two ranks both come from the same rank, in put order)
            w, r = self.w, self.rank
            lower, upper = (r - 1) % w.world, (r + 1) % w.world
            w.q[(r, upper)].put(("to_upper", to_upper))
            w.q[(r, lower)].put(("to_lower", to_lower))
            if lower == upper:
                msgs = dict(w.q[(lower, r)].get(timeout=120) for _ in range(2))
            else:
                msgs = dict([w.q[(lower, r)].get(timeout=120), w.q[(upper, r)].get(timeout=120)])
            return msgs["to_upper"], msgs["to_lower"]

        def _gather(self, x):
            w = self.w
            w.slots[self.rank] = np.asarray(x, np.float64).copy()
            w.barrier.wait(timeout=120)
            out = [s.copy() for s in w.slots]
            w.barrier.wait(timeout=120)
            return out

        def allreduce_sum(self, x):
            return np.sum(self._gather(x), axis=0)

        def allgather(self, x):
            return self._gather(x)

    def run(self, fn):
        res = [None] * self.world
        err = []

        def go(r):
            try:
                res[r] = fn(r, ThreadWorld._Comm(self, r))
            except BaseException as e:  # noqa: BLE001 -- re-raised below
                err.append(e)
                self.barrier.abort()

        th = [threading.Thread(target=go, args=(r,)) for r in range(self.world)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        if err:
            raise err[0]
        return res


# ---------------------------------------------------------------------------
# a slab in the library's kernels
# ---------------------------------------------------------------------------
class SlabLattice:
    """One slab as a Lattice (torch device memory) of extents (N0, N1, N2,
    n + 2) whose draws are the whole lattice's.  Its links are set from the
    slab's local configuration; class slices are contiguous in the link
    store (a class holds its V/2 links ordered by half-site index, time
    slowest), so get_slice returns a device view and set_slice copies into
    one, on the lattice's stream."""

    def __init__(self, geom, beta, seed=1, prec="f64", U_local=None, stream=None):
        import torch
        from .lattice import Lattice
        self.geom = geom
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.prec = prec
        with torch.cuda.stream(self.stream):
            self.lat = Lattice(geom.local_dims, beta, seed=seed, start="cold", prec=prec, stream=self.stream)
            self.lat.set_site_offset(geom.site0)
            self.lat.set_schedule("substep")
            if U_local is not None:
                self.lat.set_links(U_local)
        self.lb = {"f64": 32, "f32": 16, "f16q": 8}[prec]
        self.vh = geom.nsig * (geom.n + 2) // 2
        self.hs = geom.nsig // 2

    def _view(self, t, mu, p):
        cls = 2 * mu + p
        off = (cls * self.vh + t * self.hs) * self.lb
        return self.lat._buf[off:off + self.hs * self.lb]

    def substep(self, mu, p_local, sweep_index):
        self.lat.substep(mu, p_local, sweep_index)

    def get_slice(self, t, mu, p):
        import torch
        with torch.cuda.stream(self.stream):
            out = self._view(t, mu, p).clone()
        self.stream.synchronize()   # ready for a copy on another rank's stream
        return out

    def set_slice(self, t, mu, p, data):
        import torch
        with torch.cuda.stream(self.stream):
            d = torch.as_tensor(data)
            self._view(t, mu, p).copy_(d.to(self._view(t, mu, p).device, non_blocking=False))

    def plaquette_slices(self, t_first, t_count):
        return self.lat.plaquette_slices(t_first, t_count)

    def time_lines(self, t_first, t_count):
        return self.lat.time_lines(t_first, t_count)

    def own_links(self):
        return self.geom.own_part(self.lat.get_links())

    def close(self):
        self.lat.close()
