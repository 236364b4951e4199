"""The time-slab decomposition with the library's kernels (SlabLattice) on
one GPU.  The slabs run as host threads of one process, each on its own
stream; their ghost slices move through host queues, so no kernel waits on
another.  After two sweeps the slabs' own links must equal those of the
undivided lattice bit for bit (the slab's Philox site offset makes its draws
the whole lattice's), and the plaquette and Polyakov loop combined across
slabs must equal the undivided lattice's up to the order of summation.
"""
import numpy as np
import pytest

from paper_1010_4834_gb300 import Lattice, tslab

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-6)])
@pytest.mark.parametrize("world", [1, 2, 4])
def test_slabs_run_the_undivided_lattice(world, prec, tol):
    import torch
    dims, beta, seed = (8, 6, 4, 16), 2.4, 13
    whole = Lattice(dims, beta, seed=seed, start="hot", prec=prec)
    U0 = whole.get_links()
    whole.sweep(2)
    U = whole.get_links()
    P, L = whole.plaquette(), whole.polyakov()
    whole.close()

    def rank(r, comm):
        torch.cuda.set_device(0)
        geom = tslab.SlabGeometry(dims, world, r)
        store = tslab.SlabLattice(geom, beta, seed=seed, prec=prec, U_local=geom.local_config(U0))
        for sw in range(2):
            tslab.sweep(store, comm, geom, sw)
        out = store.own_links(), tslab.plaquette(store, comm, geom), tslab.polyakov(store, comm, geom)
        store.close()
        return out

    res = tslab.ThreadWorld(world).run(rank)
    np.testing.assert_array_equal(np.concatenate([r[0] for r in res], axis=0), U)
    for _, p, l in res:
        np.testing.assert_allclose(p, P, rtol=0, atol=tol)
        assert abs(l - L) < tol
