"""The time-slab decomposition (paper_1010_4834_gb300/tslab.py) on the CPU.

Each slab runs its substeps with the oracle (a store defined here: the
oracle's staple on the slab's ghosted local lattice and its heat-bath draw
with the whole lattice's site index), so the decomposition, the parity
mapping, the Philox site offset and the ghost exchange are checked without a
GPU: after two sweeps the slabs' own links must equal the undivided oracle
chain's bit for bit, and the plaquette (all-reduce of the slabs' sums) and
the Polyakov loop (time lines multiplied across slabs) must equal the
oracle's.  Ranks run as threads of one process (1, 2 and 4 slabs) and as two
gloo processes.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import su2mat
from paper_1010_4834_gb300 import tslab

DIMS = (4, 4, 4, 8)
BETA = 2.3
SEED = 11


class OracleSlabStore:
    """A slab whose arithmetic is the oracle's (test infrastructure)."""

    def __init__(self, geom, U_local, ch):
        self.g, self.U, self.ch = geom, np.array(U_local, copy=True), ch
        d = geom.local_dims
        s = np.arange(int(np.prod(d)))
        x = su2mat.coords(d, s)
        self.par = (x[0] + x[1] + x[2] + x[3]) & 1
        self.t = x[3]
        self.sh = su2mat.shift_table(d)

    def substep(self, mu, p_local, sweep_index):
        own = (self.t >= 1) & (self.t <= self.g.n) & (self.par == p_local)
        for s in np.flatnonzero(own):
            sig = oracle.staple(list(self.g.local_dims), self.U, int(s), mu)
            s_global = (int(s) + self.g.site0) % (1 << 32)
            _, new, _ = oracle.heatbath_link(self.ch, s_global, mu, sweep_index, sig, self.U[s, mu])
            self.U[s, mu] = new

    def _idx(self, t, p):
        return np.flatnonzero((self.t == t) & (self.par == p))

    def get_slice(self, t, mu, p):
        return self.U[self._idx(t, p), mu].copy()

    def set_slice(self, t, mu, p, data):
        self.U[self._idx(t, p), mu] = np.asarray(data)

    def plaquette_slices(self, t_first, t_count):
        # (1/2) Re Tr of the plaquettes based at the sites of these slices, in
        # 2x2 matrices (su2mat), means over 3 nsig t_count plaquettes per part
        sel = np.flatnonzero((self.t >= t_first) & (self.t < t_first + t_count))
        M = su2mat.to_mat(self.U)
        ss = ts = 0.0
        for mu in range(4):
            for nu in range(mu + 1, 4):
                a = M[sel, mu] @ M[self.sh[sel, mu, 0], nu]
                b = M[sel, nu] @ M[self.sh[sel, nu, 0], mu]
                v = su2mat.half_retr(a @ su2mat.dag(b)).sum()
                if nu == 3:
                    ts += v
                else:
                    ss += v
        n3 = 3.0 * len(sel)
        return np.array([(ss + ts) / (2 * n3), ss / n3, ts / n3])

    def time_lines(self, t_first, t_count):
        nsig = self.g.nsig
        M = su2mat.to_mat(self.U)
        pr = np.broadcast_to(su2mat.ONE, (nsig, 2, 2)).copy()
        for t in range(t_first, t_first + t_count):
            pr = pr @ M[t * nsig:(t + 1) * nsig, 3]
        return su2mat.to_quat(pr)

    def own_links(self):
        return self.g.own_part(self.U)


def reference(nsweeps):
    ch = oracle.chain(BETA, seed=SEED)
    U0 = oracle.init_hot(list(DIMS), ch)
    U = U0.copy()
    for sw in range(nsweeps):
        oracle.sweep(list(DIMS), U, ch, sw)
    return U0, U, oracle.plaquette(list(DIMS), U), oracle.polyakov(list(DIMS), U)


def run_rank(rank, comm, world, U0, nsweeps):
    geom = tslab.SlabGeometry(DIMS, world, rank)
    store = OracleSlabStore(geom, geom.local_config(U0), oracle.chain(BETA, seed=SEED))
    for sw in range(nsweeps):
        tslab.sweep(store, comm, geom, sw)
    return store.own_links(), tslab.plaquette(store, comm, geom), tslab.polyakov(store, comm, geom)


@pytest.mark.parametrize("world", [1, 2, 4])
def test_slabs_as_threads_run_the_undivided_chain(world):
    U0, U, P, L = reference(2)
    res = tslab.ThreadWorld(world).run(lambda r, comm: run_rank(r, comm, world, U0, 2))
    links = np.concatenate([r[0] for r in res], axis=0)
    np.testing.assert_array_equal(links, U)
    for _, p, l in res:
        np.testing.assert_allclose(p, P, rtol=0, atol=1e-13)
        assert abs(l - L) < 1e-13


def test_geometry_rules():
    g = tslab.SlabGeometry((4, 4, 4, 8), 2, 1)
    assert g.n == 4 and g.t0 == 4 and g.local_dims == (4, 4, 4, 6)
    assert g.site0 == 3 * 64 and g.global_slice(0) == 3 and g.global_slice(5) == 0
    assert tslab.SlabGeometry((4, 4, 4, 8), 2, 0).site0 == (1 << 32) - 64     # slice -1 wraps
    for bad in ((4, 4, 4, 6), (4, 4, 4, 8, 3)):
        with pytest.raises(ValueError):
            tslab.SlabGeometry(bad[:4], bad[4] if len(bad) > 4 else 4, 0)
    # the ghosted local configuration holds the neighbours' boundary slices
    U = np.arange(np.prod((4, 4, 4, 8)) * 16, dtype=float).reshape(-1, 4, 4)
    loc = g.local_config(U)
    np.testing.assert_array_equal(loc[:64], U[3 * 64:4 * 64])
    np.testing.assert_array_equal(loc[5 * 64:], U[0:64])
    np.testing.assert_array_equal(g.own_part(loc), U[4 * 64:8 * 64])


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, world, port, U0, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    comm = tslab.TorchComm()
    links, p, l = run_rank(rank, comm, world, U0, 2)
    out[rank] = (links.tobytes(), p.tolist(), l)
    dist.destroy_process_group()


def test_slabs_as_gloo_ranks_run_the_undivided_chain():
    world = 2
    U0, U, P, L = reference(2)
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_gloo_rank, args=(r, world, port, U0, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
            assert p.exitcode == 0
        res = [out[r] for r in range(world)]
    links = np.concatenate([np.frombuffer(r[0]).reshape(-1, 4, 4) for r in res], axis=0)
    np.testing.assert_array_equal(links, U)
    for _, p, l in res:
        np.testing.assert_allclose(p, P, rtol=0, atol=1e-13)
        assert abs(l - L) < 1e-13
