"""The fused parity-pair schedule (su2_set_schedule "pair", su2_heatbath_pair)
and interleaved over-relaxation (su2_set_overrelax).

Both halves of a pair run the same per-link code as the substep kernel and
every draw is keyed by (sweep, site, direction), so the pair schedule must
leave the links of the substep schedule bit for bit -- on every shape (time
extents down to 2, slices smaller than one work chunk, ragged chunks), every
branch of the update and both graph and direct launches.  The substep
schedule is itself checked against the oracle link by link
(test_gpu_parity.py), and the 64^4 measured-sweep test there runs the pair.
"""
import numpy as np
import pytest

import oracle
from paper_1010_4834_gb300 import Batch, Lattice, SU2Error, inputs, kernel_launches

pytestmark = pytest.mark.gpu

SHAPES = [(2, 2, 2, 2), (4, 4, 4, 4), (6, 4, 2, 10), (8, 6, 4, 10), (12, 10, 8, 6), (4, 4, 4, 64),
          (16, 16, 16, 16), (32, 32, 32, 4), (34, 18, 20, 12)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def pair_and_substep(dims, prec, beta, seed, max_tries=64, sampler="kp"):
    a = Lattice(dims, beta, seed=seed, start="hot", prec=prec)
    b = Lattice(dims, beta, seed=seed, start="hot", prec=prec)
    a.set_schedule("pair")
    b.set_schedule("substep")
    for lat in (a, b):
        lat.set_options(max_tries, sampler)
    return a, b


@pytest.mark.parametrize("prec", ["f32", "f16q"])
@pytest.mark.parametrize("dims", SHAPES)
def test_pair_schedule_leaves_the_substep_links(dims, prec):
    a, b = pair_and_substep(dims, prec, 2.3, 5)
    a.sweep(3)                   # direct launches
    b.sweep(3)
    np.testing.assert_array_equal(a.get_links(), b.get_links())
    a.sweep(9)                   # one graph replay of eight sweeps, then one more
    b.sweep(9)
    np.testing.assert_array_equal(a.get_links(), b.get_links())
    ha = a.sweep_measure(10)     # measured: the parity-1 half sums the plaquette
    hb = b.sweep_measure(10)
    np.testing.assert_array_equal(a.get_links(), b.get_links())
    np.testing.assert_array_equal(ha[:, 3], hb[:, 3])
    # the same plaquette, summed in another order (FP32 per-thread sums)
    np.testing.assert_allclose(ha[:, :3], hb[:, :3], rtol=0, atol=2e-6)
    np.testing.assert_allclose(ha[-1, :3], a.plaquette(), rtol=0, atol=2e-6)
    assert a.sweep_count == b.sweep_count == 22
    a.close()
    b.close()


@pytest.mark.parametrize("beta,max_tries,sampler", [
    (0.4, 64, "kp"),     # low acceptance: most links go through the deferral queue
    (0.0, 64, "kp"),     # alpha = 0: Haar links
    (2.3, 1, "kp"),      # capped links keep their old value
    (2.3, 3, "creutz"),
    (0.05, 64, "kp"),    # many links exhaust their trials
])
@pytest.mark.parametrize("dims", [(8, 6, 4, 10), (16, 16, 16, 16)])
def test_pair_schedule_every_branch(dims, beta, max_tries, sampler):
    a, b = pair_and_substep(dims, "f32", beta, 9, max_tries, sampler)
    ha = a.sweep_measure(4)
    hb = b.sweep_measure(4)
    np.testing.assert_array_equal(a.get_links(), b.get_links())
    np.testing.assert_array_equal(ha[:, 3], hb[:, 3])
    np.testing.assert_allclose(ha[:, :3], hb[:, :3], rtol=0, atol=3e-6)
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["f32", "f16q"])
def test_single_pair_call_against_the_oracle(prec):
    # su2_heatbath_pair(mu) = substeps (mu, 0) then (mu, 1) of one sweep
    # index.  Each half is compared with the oracle's substep from the state
    # that half saw: the start for parity 0, and for parity 1 the final links
    # with the parity-1 MU links put back to their start values (parity 1
    # changes nothing else).  Links whose accept decision is within rounding
    # of flipping are checked for validity only, as in the substep test.
    dims = (8, 6, 4, 10)
    U0 = inputs.random_field(dims, 77)
    V = int(np.prod(dims))
    s = np.arange(V)
    par = (s % dims[0] + s // dims[0] % dims[1] + s // (dims[0] * dims[1]) % dims[2]
           + s // (dims[0] * dims[1] * dims[2])) & 1
    tol = {"f32": 2e-5, "f16q": 4e-3}[prec]
    for mu in range(4):
        lat = Lattice(dims, 2.3, seed=7, prec=prec)
        lat.set_links(U0)
        start = lat.get_links()
        lat.pair(mu, 11)
        got = lat.get_links()
        lat.close()
        ch = oracle.chain(2.3, seed=7, u23=1)
        checked = 0
        for p in (0, 1):
            ref = start.copy() if p == 0 else got.copy()
            if p == 1:
                ref[par == 1, mu] = start[par == 1, mu]
            _, m = oracle.substep(list(dims), ref, ch, 11, mu, p, margins=True)
            ok = (par == p) & (m[:, mu] >= 1e-4)
            diff = np.abs(got[:, mu] - ref[:, mu]).max(axis=-1)
            assert (diff[ok] < tol).all(), (mu, p, diff[ok].max())
            checked += ok.sum()
        assert checked > 0.99 * V
        # nothing outside class mu moved
        others = [d for d in range(4) if d != mu]
        np.testing.assert_array_equal(got[:, others], start[:, others])


def test_pair_schedule_arguments_and_launch_count():
    with pytest.raises(SU2Error):
        Lattice((4, 4, 4, 4), 2.0, prec="f64").set_schedule("pair")
    lat = Lattice((4, 4, 6, 4), 2.3, seed=5, start="hot", prec="f32")
    with pytest.raises(SU2Error):
        lat.set_schedule(7)
    with pytest.raises(SU2Error):
        lat.set_overrelax(17)
    lat.set_schedule("pair")
    n0 = kernel_launches()
    lat.sweep_measure(6)
    assert kernel_launches() - n0 == 6 * (4 + 1)      # four pairs and the Polyakov kernel
    lat.set_overrelax(2)
    n0 = kernel_launches()
    lat.sweep_measure(16)                              # two graph replays
    assert kernel_launches() - n0 == 16 * (2 * 8 + 4 + 1)
    lat.close()


@pytest.mark.parametrize("schedule,prec", [("substep", "f64"), ("pair", "f32")])
def test_overrelaxation_before_each_heatbath_sweep(schedule, prec):
    # with n over-relaxation sweeps per heat-bath sweep, a sweep is n oracle
    # over-relaxation sweeps followed by the oracle's heat-bath sweep; the
    # measured sweep's plaquette (from the heat bath's staples) is that of
    # the final links
    # (from a configuration thermalised by ten heat-bath sweeps: on the
    # random hot start, small staples magnify the rounding of the reflection)
    dims = (4, 6, 4, 8)
    lat = Lattice(dims, 2.4, seed=3, start="hot", prec=prec)
    lat.set_schedule(schedule)
    lat.sweep(10)
    lat.set_overrelax(2)
    ch = oracle.chain(2.4, seed=3, u23=0 if prec == "f64" else 1)
    U = lat.get_links()
    hist = lat.sweep_measure(2)
    for sw in range(10, 12):
        for _ in range(2):
            for mu in range(4):
                for p in range(2):
                    oracle.overrelax_substep(list(dims), U, mu, p)
        oracle.sweep(list(dims), U, ch, sw)
    got = lat.get_links()
    if prec == "f64":
        assert np.abs(got - U).max() < 1e-12
        np.testing.assert_allclose(hist[-1, :3], oracle.plaquette(list(dims), U), rtol=0, atol=1e-12)
    else:
        # FP32: after two sweeps a few decisions may have flipped; nearly all
        # links agree to FP32 accuracy
        assert (np.abs(got - U).max(axis=-1) < 2e-5).mean() > 0.98
        np.testing.assert_allclose(hist[-1, :3], lat.plaquette(), rtol=0, atol=2e-6)
    lat.close()


def test_batched_overrelaxation_before_each_heatbath_sweep():
    # the batched kernel with one over-relaxation sweep before each heat-bath
    # sweep, lattice by lattice against the oracle (FP64)
    dims = [(4, 4, 4, 4), (6, 4, 4, 2)]
    betas = [2.2, 2.5]
    b = Batch(dims, betas, seed=19, start="hot", prec="f64")
    start = []
    for i, d in enumerate(dims):
        # a configuration thermalised by the oracle (ten heat-bath sweeps)
        ch = oracle.chain(betas[i], seed=91, lattice_id=i)
        U = oracle.init_hot(list(d), ch)
        for sw in range(10):
            oracle.sweep(list(d), U, ch, sw)
        start.append(U)
        b.set_links(i, U)
    b.set_overrelax(1)
    b.sweep(2)
    for i, d in enumerate(dims):
        ch = oracle.chain(betas[i], seed=19, lattice_id=i)
        U = start[i].copy()
        for sw in range(2):
            for mu in range(4):
                for p in range(2):
                    oracle.overrelax_substep(list(d), U, mu, p)
            oracle.sweep(list(d), U, ch, sw)
        assert np.abs(b.get_links(i) - U).max() < 1e-12
    with pytest.raises(SU2Error):
        b.set_overrelax(-1)
    b.close()
