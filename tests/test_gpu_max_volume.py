"""The largest lattice the library accepts: 256^3 x 126 = 2,113,929,216 sites,
just below the 2^31 - 1 site limit, in F16Q (links 68 GB, with the two APE
buffers 169 GB of device memory).  Hot start and one heat-bath substep,
checked on sampled sites (including the last ones) against the oracle: each
sampled site's 3^4 neighbourhood is copied out with su2_get_sites into a small
4^4 lattice, where the oracle evaluates the same staple (every link it reads
lies within one step of the site, so the small lattice never wraps)."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1010_4834_gb300 import Lattice
from paper_1010_4834_gb300.lattice import required_bytes

pytestmark = pytest.mark.gpu

DIMS = (256, 256, 256, 126)
V = 256 ** 3 * 126


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def coords(s):
    x = []
    for n in DIMS:
        x.append(s % n)
        s //= n
    return x


def index(x):
    s = 0
    for c, n in zip(reversed(x), reversed(DIMS)):
        s = s * n + c % n
    return s


def neighbourhood(lat, s):
    """4^4 canonical field holding the links of the 3^4 sites around s, with
    s at local (1, 1, 1, 1); the rest is the identity."""
    U = np.zeros((4 ** 4, 4, 4))
    U[:, :, 0] = 1.0
    x = coords(s)
    for d in itertools.product((-1, 0, 1), repeat=4):
        y = index([x[i] + d[i] for i in range(4)])
        loc = (1 + d[0]) + 4 * ((1 + d[1]) + 4 * ((1 + d[2]) + 4 * (1 + d[3])))
        U[loc] = lat.get_sites(y, 1)[0]
    return U


def test_maximum_volume_hot_start_and_substep():
    import torch
    assert V < 2 ** 31 - 1
    need = required_bytes(DIMS, "f16q")
    free, _ = torch.cuda.mem_get_info()
    if free < need + (4 << 30):
        pytest.skip("needs %.0f GB of free device memory" % (need / 1e9))
    beta, mu, parity = 2.6, 1, 1
    lat = Lattice(DIMS, beta, seed=5, start="hot", prec="f16q")
    ch = oracle.chain(beta, seed=5, u23=1)
    rng = np.random.default_rng(3)
    sample = [0, 1, V - 2, V - 1, 2 ** 31 - 2 ** 25] + [int(s) for s in rng.integers(0, V, 40)]
    sample = [s for s in sample if s < V]
    for s in sample:
        got = lat.get_sites(s, 1)[0]
        for m in range(4):
            assert np.abs(got[m] - oracle.hot_link(ch, s, m)).max() < 2e-3, (s, m)
    odd = [s for s in sample if sum(coords(s)) % 2 == parity]
    assert V - 2 in odd
    before = {s: neighbourhood(lat, s) for s in odd}
    lat.substep(mu, parity, 0)
    checked = 0
    centre = 1 + 4 * (1 + 4 * (1 + 4 * 1))
    for s in odd:
        U0 = before[s]
        after = lat.get_sites(s, 1)[0]
        np.testing.assert_array_equal(after[[0, 2, 3]], U0[centre, [0, 2, 3]])
        sig = oracle.staple([4, 4, 4, 4], U0, centre, mu)
        n, new, margin = oracle.heatbath_link(ch, s, mu, 0, sig, U0[centre, mu])
        if margin < 1e-4:
            continue
        assert np.abs(after[mu] - new).max() < 2e-3, (s, after[mu], new)
        checked += 1
    assert checked >= 15
    even = [s for s in sample if sum(coords(s)) % 2 != parity]
    for s in even[:5]:
        assert np.abs(lat.get_sites(s, 1)[0][mu] - oracle.hot_link(ch, s, mu)).max() < 2e-3
    # plaquette reduction over 12.7e9 plaquettes: on the hot start every plane
    # averages to 0 (within 1e-4); after the substep only the planes (1, nu)
    # moved, each plaquette of them holding exactly one new link, so the
    # spatial mean (two such planes of three) is twice the space-time mean
    # (one of three), and both are positive
    p = lat.plaquette()
    assert np.all(np.isfinite(p))
    assert abs(p[0] - 0.5 * (p[1] + p[2])) < 1e-12
    assert 0.05 < p[2] < 0.2
    assert abs(p[1] - 2 * p[2]) < 2e-3
    lat.close()
