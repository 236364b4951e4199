"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Same seeded inputs on both sides; comparisons element by element.
Tolerances:
  * FP64 links: 1e-12 absolute per quaternion component (the heat-bath
    per-link bar).  Rounding differs only in the order of a few FP64
    operations and in libm vs CUDA transcendentals (both within a few ulp).
  * FP32 links: 2e-5 absolute.  A binary32 heat-bath update carries a few
    ulp (6e-8) of error per operation through ~100 dependent operations;
    links whose accept/reject decision the oracle finds within 1e-4 of
    flipping are compared only for validity (unit norm), since either
    outcome is a correct draw.
  * F16Q storage: 4e-3 absolute (binary16 rounding, 2^-11 relative, of each
    component before the FP32 renormalisation on load).
  * Measurements: FP64 1e-12, FP32 2e-6 absolute (means of values in [-1,1]).
"""
import os

import numpy as np
import pytest

import oracle
from paper_1010_4834_gb300 import Batch, Lattice, SU2Error, inputs

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-5, "f16q": 4e-3}
MTOL = {"f64": 1e-12, "f32": 2e-6, "f16q": 2e-3}
SHAPES = [(2, 2, 2, 2), (4, 4, 4, 4), (6, 4, 2, 10), (8, 8, 8, 8), (4, 6, 8, 2)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def u23(prec):
    return 0 if prec == "f64" else 1


def as_stored(U, prec):
    """The values a store of this precision holds for U (what set_links keeps)."""
    if prec == "f32":
        return U.astype(np.float32).astype(np.float64)
    if prec == "f16q":
        q = U.astype(np.float16).astype(np.float64)
        return q / np.linalg.norm(q, axis=-1, keepdims=True)
    return U.copy()


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["f64", "f32", "f16q"])
@pytest.mark.parametrize("dims", SHAPES)
def test_start_configurations(dims, prec):
    lat = Lattice(dims, 2.0, seed=5, start="cold", prec=prec)
    U = lat.get_links()
    assert np.array_equal(U, oracle.init_cold(list(dims)))
    lat.close()
    lat = Lattice(dims, 2.0, seed=0x123456789, start="hot", prec=prec)
    ch = oracle.chain(2.0, seed=0x123456789, u23=u23(prec))
    ref = oracle.init_hot(list(dims), ch)
    got = lat.get_links()
    assert np.abs(got - ref).max() < {"f64": 1e-14, "f32": 2e-6, "f16q": 4e-3}[prec]
    lat.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "f16q"])
def test_set_get_roundtrip(prec):
    dims = (4, 6, 2, 8)
    U = inputs.random_field(dims, 3)
    lat = Lattice(dims, 2.0, prec=prec)
    lat.set_links(U)
    got = lat.get_links()
    if prec == "f64":
        assert np.array_equal(got, U)
    elif prec == "f32":
        assert np.array_equal(got, as_stored(U, prec))
    else:
        # binary16 storage; the FP32 renormalisation on load adds ~1 ulp
        assert np.abs(got - as_stored(U, prec)).max() < 5e-7
    lat.close()


@pytest.mark.parametrize("prec", ["f64", "f16q"])
def test_pinned_host_buffers_take_the_direct_path(prec):
    # a page-locked source is read by the conversion kernel directly; the
    # result must equal the staged copy of pageable memory, and reading back
    # into page-locked buffers (whole and a site range) must agree too
    import torch
    dims = (8, 6, 4, 10)
    U = inputs.random_field(dims, 17)
    V = int(np.prod(dims))
    pinned = torch.from_numpy(U.copy()).pin_memory()
    a = Lattice(dims, 2.0, prec=prec)
    b = Lattice(dims, 2.0, prec=prec)
    a.set_links(pinned.numpy())
    b.set_links(U)
    out = torch.empty((V, 4, 4), dtype=torch.float64).pin_memory()
    a.get_links(out.numpy())
    np.testing.assert_array_equal(out.numpy(), b.get_links())
    part = torch.empty((100, 4, 4), dtype=torch.float64).pin_memory()
    from paper_1010_4834_gb300 import _lib
    from paper_1010_4834_gb300.lattice import _dptr
    _lib.check(_lib.load().su2_get_sites(a._h, 777, 100, _dptr(part.numpy())))
    np.testing.assert_array_equal(part.numpy(), b.get_sites(777, 100))
    a.close()
    b.close()


def test_set_links_from_device_memory():
    # a float64 CUDA tensor in the canonical layout is read on the device by
    # the conversion kernel; the result equals the host path bit for bit
    import torch
    dims = (8, 6, 4, 10)
    U = inputs.random_field(dims, 23)
    for prec in ("f64", "f32", "f16q"):
        a = Lattice(dims, 2.0, prec=prec)
        b = Lattice(dims, 2.0, prec=prec)
        d = torch.from_numpy(U.copy()).cuda()
        torch.cuda.current_stream().synchronize()
        a.set_links(d)
        b.set_links(U)
        np.testing.assert_array_equal(a.get_links(), b.get_links())
        a.close()
        b.close()


# ---------------------------------------------------------------------------
def substep_compare(dims, prec, beta, U0, mu, p, sweep, sampler="kp", max_tries=64, seed=7):
    lat = Lattice(dims, beta, seed=seed, prec=prec)
    lat.set_options(max_tries, sampler)
    lat.set_links(U0)
    lat.substep(mu, p, sweep)
    got = lat.get_links()
    lat.close()
    ref = as_stored(U0, prec)
    ch = oracle.chain(beta, seed=seed, max_tries=max_tries,
                      sampler=oracle.KP if sampler == "kp" else oracle.CREUTZ, u23=u23(prec))
    st, marg = oracle.substep(list(dims), ref, ch, sweep, mu, p, margins=True)
    ok = marg[:, mu] >= (0 if prec == "f64" else 1e-4)
    diff = np.abs(got - ref).max(axis=-1)          # (V, 4)
    bad = np.argwhere((diff > TOL[prec]) & ok[:, None])
    assert len(bad) == 0, (prec, dims, mu, p, len(bad), diff.max())
    # undecided links are still valid SU(2) elements
    n = np.linalg.norm(got.reshape(-1, 4), axis=-1)
    assert np.abs(n - 1).max() < (1e-12 if prec == "f64" else 1e-5 if prec == "f32" else 2e-3)
    return st, (~ok).sum()


@pytest.mark.parametrize("prec", ["f64", "f32", "f16q"])
@pytest.mark.parametrize("dims", SHAPES)
def test_heatbath_substep(dims, prec):
    U0 = inputs.random_field(dims, 11)
    undecided = 0
    for mu in range(4):
        for p in range(2):
            _, u = substep_compare(dims, prec, 2.3, U0, mu, p, sweep=3 + mu)
            undecided += u
    assert undecided <= max(2, 0.002 * np.prod(dims) * 4)


@pytest.mark.parametrize("sampler,max_tries,beta", [("creutz", 64, 1.7), ("kp", 1, 2.0), ("kp", 3, 0.3),
                                                    ("kp", 64, 0.0), ("creutz", 2, 6.0)])
def test_heatbath_sampler_options(sampler, max_tries, beta):
    dims = (4, 4, 6, 4)
    U0 = inputs.random_field(dims, 12)
    st, _ = substep_compare(dims, "f64", beta, U0, 2, 1, sweep=9, sampler=sampler, max_tries=max_tries)
    if beta == 0.0:
        assert st.haar == st.updates
    if max_tries == 1:
        assert st.capped > 0                       # keep-old path exercised


@pytest.mark.parametrize("start", ["cold", "hot"])
def test_sweep_parity_fp64(start):
    """Config: 8^4, beta = 2.4, seed 1: one and two full sweeps, per link 1e-12."""
    dims = (8, 8, 8, 8)
    lat = Lattice(dims, 2.4, seed=1, start=start, prec="f64")
    ch = oracle.chain(2.4, seed=1)
    U = oracle.init_hot(list(dims), ch) if start == "hot" else oracle.init_cold(list(dims))
    for sw in range(2):
        lat.sweep(1)
        oracle.sweep(list(dims), U, ch, sw)
        got = lat.get_links()
        assert np.abs(got - U).max() < 1e-12, (start, sw, np.abs(got - U).max())
    assert lat.sweep_count == 2
    np.testing.assert_allclose(lat.plaquette(), oracle.plaquette(list(dims), U), atol=1e-12, rtol=0)
    assert abs(lat.polyakov() - oracle.polyakov(list(dims), U)) < 1e-12
    lat.close()


def test_config_8x4_cold_fp64_hundred_sweeps_against_oracle():
    """8^4, beta 2.4, cold start, seed 1, FP64: 100 measured sweeps.  With the
    same Philox stream the GPU chain follows the oracle's trajectory through
    1.6 M updates: no accept decision flips, and the plaquette and Polyakov
    loop after every sweep agree while the rounding differences (1e-16 at the
    first sweep) grow through the chaotic dynamics to a few 1e-9 by sweep 100."""
    dims = (8, 8, 8, 8)
    lat = Lattice(dims, 2.4, seed=1, start="cold", prec="f64")
    hist = lat.sweep_measure(100)
    got = lat.get_links()
    lat.close()
    ch = oracle.chain(2.4, seed=1)
    U = oracle.init_cold(list(dims))
    ref = np.empty((100, 4))
    for sw in range(100):
        oracle.sweep(list(dims), U, ch, sw)
        ref[sw, :3] = oracle.plaquette(list(dims), U)
        ref[sw, 3] = oracle.polyakov(list(dims), U)
    np.testing.assert_allclose(hist[:10], ref[:10], atol=1e-13, rtol=0)
    np.testing.assert_allclose(hist, ref, atol=1e-7, rtol=0)
    assert np.abs(got - U).max() < 1e-5


def test_graph_replay_matches_single_sweeps():
    dims = (4, 4, 4, 8)
    a = Lattice(dims, 2.2, seed=3, start="hot", prec="f64")
    b = Lattice(dims, 2.2, seed=3, start="hot", prec="f64")
    a.sweep(19)                      # two graph replays of 8 + 3 direct sweeps
    for _ in range(19):
        b.sweep(1)
    assert a.sweep_count == b.sweep_count == 19
    assert np.array_equal(a.get_links(), b.get_links())
    a.close()
    b.close()


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["f64", "f32", "f16q"])
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 6, 2, 8), (6, 4, 4, 10)])
def test_measurements(dims, prec):
    U = inputs.random_field(dims, 21)
    lat = Lattice(dims, 2.0, prec=prec)
    lat.set_links(U)
    ref = as_stored(U, prec)
    np.testing.assert_allclose(lat.plaquette(), oracle.plaquette(list(dims), ref), atol=MTOL[prec], rtol=0)
    assert abs(lat.polyakov() - oracle.polyakov(list(dims), ref)) < MTOL[prec]
    rmax, tmax = min(dims[:3]), dims[3]
    np.testing.assert_allclose(lat.wilson_loops(rmax, tmax), oracle.wilson_loops(list(dims), ref, rmax, tmax),
                               atol=MTOL[prec] * 5, rtol=0)
    lat.close()


# Long time extents: each time line is split over a group of up to 32 lanes
# (segments of >= 8 links) whose products are combined by shuffles in t
# order.  nt = 16 .. 256 covers 2 .. 32 lanes, segments with a ragged chunk
# (40: 4 x 10) and odd segment lengths (18: 2 x 9, 36: 4 x 9), where half
# the segments start on an odd t.  Random fields: an out-of-order product
# changes every line's trace.
@pytest.mark.parametrize("prec", ["f64", "f32", "f16q"])
@pytest.mark.parametrize("nt", [16, 18, 24, 36, 40, 64, 256])
def test_polyakov_long_time_extent(nt, prec):
    dims = (2, 4, 2, nt)
    U = inputs.random_field(dims, 31 + nt)
    lat = Lattice(dims, 2.0, prec=prec)
    lat.set_links(U)
    ref = as_stored(U, prec)
    assert abs(lat.polyakov() - oracle.polyakov(list(dims), ref)) < MTOL[prec]
    lat.close()


def test_measurements_on_thermalised_configuration():
    dims = (8, 8, 8, 8)
    lat = Lattice(dims, 2.5, seed=2, start="hot", prec="f64")
    lat.sweep(20)
    U = lat.get_links()
    np.testing.assert_allclose(lat.plaquette(), oracle.plaquette(list(dims), U), atol=1e-12, rtol=0)
    assert abs(lat.polyakov() - oracle.polyakov(list(dims), U)) < 1e-12
    np.testing.assert_allclose(lat.wilson_loops(8, 8), oracle.wilson_loops(list(dims), U, 8, 8), atol=1e-12)
    lat.close()


# Wilson loops across the kernels' limits: R and T up to 16 with Nt / 8 in
# {1, 2, 4, 6, 8} run the temporal-gauge kernel (R = 16 here, lines that wrap
# several times around a row); other time extents, R = 17 or T > 16 the
# time-outer kernel (R = 17 needs its second register chunk, which starts
# from prefix products; T = 18, 20 a second T chunk); planes too large for
# shared memory fall back to the time-outer kernel's bands or the
# global-memory kernel.
_WILSON_REF = {}


@pytest.mark.parametrize("prec", ["f32", "f16q", "f64"])
@pytest.mark.parametrize("dims,rmax,tmax", [((18, 18, 18, 4), 17, 4), ((12, 12, 12, 4), 12, 4),
                                            ((4, 4, 4, 18), 4, 18), ((6, 10, 8, 6), 6, 6),
                                            ((16, 16, 16, 8), 16, 4),
                                            # temporal-gauge kernel, every row chunk it is built
                                            # for (Nt / 8 = 2, 4, 6, 8 rows a lane), time lines
                                            # wrapping past the last slice
                                            ((4, 4, 2, 16), 2, 16), ((2, 4, 2, 32), 2, 16),
                                            ((2, 2, 4, 48), 2, 16), ((2, 2, 2, 64), 2, 16),
                                            # 64-site rows with 96 slices: planes too large for
                                            # shared memory, so work units are bands of time
                                            # slices (76 / 60 slices in FP32, 30 / 14 in FP64)
                                            ((64, 2, 2, 96), 2, 16), ((64, 2, 2, 96), 2, 20),
                                            # 432- and 480-site rows: not even one time slice
                                            # (plus the lines' overhang) fits, the global-memory
                                            # kernel runs
                                            ((432, 2, 2, 16), 2, 16), ((480, 2, 2, 16), 2, 16)])
def test_wilson_loops_across_chunks(dims, rmax, tmax, prec):
    U = inputs.random_field(dims, 23)
    ref = as_stored(U, prec)
    key = (dims, rmax, tmax, prec)
    if key not in _WILSON_REF:
        _WILSON_REF[key] = oracle.wilson_loops(list(dims), ref, rmax, tmax)
    lat = Lattice(dims, 2.0, prec=prec)
    lat.set_links(U)
    np.testing.assert_allclose(lat.wilson_loops(rmax, tmax), _WILSON_REF[key], atol=MTOL[prec] * 5, rtol=0)
    lat.close()


def test_wilson_full_chunks_fp32_f16q_against_fp64_kernel():
    # W(16,16) on 32^4, the benchmark's loop range (every R up to 16, every T
    # up to 16, time lines wrapping past the last slice) in the temporal-gauge
    # kernel: FP32 / F16Q against FP64 (pinned to the oracle above) on the
    # same stored links
    dims = (32, 32, 32, 32)
    U = inputs.random_field(dims, 37)
    b = Lattice(dims, 2.0, prec="f64")
    for prec in ("f32", "f16q"):
        b.set_links(as_stored(U, prec))
        ref = b.wilson_loops(16, 16)
        a = Lattice(dims, 2.0, prec=prec)
        a.set_links(U)
        np.testing.assert_allclose(a.wilson_loops(16, 16), ref, atol=1e-5, rtol=0)
        a.close()
    b.close()


def test_wilson_loops_both_chunkings_fp32_against_fp64_kernel():
    # R and T both past their first chunk at once: the FP32 time-outer kernel
    # against the FP64 kernels (pinned to the oracle above) on one field
    dims = (18, 18, 18, 18)
    U = inputs.random_field(dims, 29)
    a = Lattice(dims, 2.0, prec="f32")
    b = Lattice(dims, 2.0, prec="f64")
    a.set_links(U)
    b.set_links(as_stored(U, "f32"))
    np.testing.assert_allclose(a.wilson_loops(17, 17), b.wilson_loops(17, 17), atol=1e-5, rtol=0)
    a.close()
    b.close()


# F16Q stores every smeared step in binary16, so it runs the short cases only
@pytest.mark.parametrize("prec,n,alpha", [(p, n, a) for p in ("f64", "f32", "f16q")
                                          for n, a in ((0, 0.7), (1, 0.7), (3, 0.444), (25, 0.7))
                                          if not (p == "f16q" and n > 3)])
@pytest.mark.parametrize("dims", [(4, 6, 4, 6), (4, 6, 4, 8)])   # time-outer and temporal-gauge kernels
def test_ape_and_smeared_wilson(prec, n, alpha, dims):
    U = inputs.random_field(dims, 31)
    lat = Lattice(dims, 2.0, prec=prec)
    lat.set_links(U)
    with pytest.raises(SU2Error):
        lat.wilson_loops(2, 2, smeared=True)      # nothing smeared yet: SU2_ESTATE
    lat.ape_smear(alpha, n)
    ref = oracle.ape_smear(list(dims), as_stored(U, prec), alpha, n)
    got = lat.wilson_loops(4, 6, smeared=True)
    exp = oracle.wilson_loops(list(dims), ref, 4, 6)
    tol = {"f64": 1e-12, "f32": 2e-5, "f16q": 5e-3}[prec]
    np.testing.assert_allclose(got, exp, atol=tol, rtol=0)
    # the chain itself is untouched
    np.testing.assert_allclose(lat.plaquette(), oracle.plaquette(list(dims), as_stored(U, prec)),
                               atol=MTOL[prec], rtol=0)
    lat.sweep(1)
    with pytest.raises(SU2Error):
        lat.wilson_loops(2, 2, smeared=True)      # a sweep invalidates the smeared copy
    lat.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "f16q"])
@pytest.mark.parametrize("dims", [(4, 4, 6, 4), (8, 6, 4, 10)])
def test_overrelaxation(dims, prec):
    # one over-relaxation sweep (Eq. 10) link by link against the oracle; the
    # update is deterministic, so every link is compared.  The input is a
    # thermalised field (ten oracle heat-bath sweeps at beta 2.4): on a random
    # field small staples magnify the rounding of W = Sigma/|Sigma| (FP32
    # reached 2e-5 there).  F16Q: each substep stores binary16 that the later
    # substeps read back, and a reflection about the staple carries those
    # 2^-12 roundings into the next links, so the oracle's output is rounded
    # to the store after every substep as well (as_stored, the storage model)
    ch = oracle.chain(2.4, seed=41)
    U = oracle.init_hot(list(dims), ch)
    for sw in range(10):
        oracle.sweep(list(dims), U, ch, sw)
    lat = Lattice(dims, 2.0, prec=prec)
    lat.set_links(U)
    lat.overrelax(1)
    ref = as_stored(U, prec)
    for mu in range(4):
        for p in range(2):
            oracle.overrelax_substep(list(dims), ref, mu, p)
            if prec == "f16q":
                ref[:, mu] = as_stored(ref[:, mu], prec)
    assert np.abs(lat.get_links() - ref).max() < TOL[prec]
    lat.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-13), ("f32", 1e-6)])
def test_overrelaxation_keeps_links_unitary_over_many_sweeps(prec, tol):
    # an over-relaxed link is built from the old one, so rounding could
    # accumulate; after 1000 sweeps every link is still a unit quaternion and
    # the action (the mean plaquette over all planes; its spatial and
    # space-time parts move) is the one before them
    dims = (8, 8, 8, 8)
    lat = Lattice(dims, 2.4, seed=7, start="hot", prec=prec)
    lat.sweep(20)
    p0 = lat.plaquette()
    lat.overrelax(1000)
    U = lat.get_links()
    assert np.abs(np.linalg.norm(U, axis=-1) - 1).max() < tol
    p1 = lat.plaquette()
    assert abs(p1[0] - p0[0]) < (1e-5 if prec == "f32" else 1e-11), (p0, p1)
    assert np.abs(p1[1:] - p0[1:]).max() > 1e-5             # the links did move
    lat.close()


# ---------------------------------------------------------------------------
def test_argument_and_state_errors():
    lat = Lattice((4, 4, 4, 4), 2.0, prec="f32")
    for bad in [lambda: lat.wilson_loops(5, 2), lambda: lat.wilson_loops(2, 5), lambda: lat.wilson_loops(0, 1),
                lambda: lat.ape_smear(1.0, 1), lambda: lat.ape_smear(0.5, -1), lambda: lat.sweep(-1),
                lambda: lat.substep(4, 0, 0), lambda: lat.set_options(0, "kp"), lambda: lat.set_beta(-1.0),
                lambda: lat.get_sites(-1, 1), lambda: lat.get_sites(250, 7), lambda: lat.layout_compare(0)]:
        with pytest.raises(SU2Error) as e:
            bad()
        assert e.value.code == 1
    with pytest.raises(SU2Error):
        Lattice((4, 4, 4, 5), 2.0)
    assert lat.get_sites(256, 0).shape == (0, 4, 4)      # an empty range at the end is valid
    lat.close()


def test_checkpoint_resume_is_bit_identical(tmp_path):
    dims = (4, 4, 4, 6)
    a = Lattice(dims, 2.3, seed=9, start="hot", prec="f64")
    a.sweep(3)
    path = tmp_path / "ck.su2"
    a.save(path)
    a.sweep(4)
    b = Lattice.load(path)
    assert b.sweep_count == 3
    b.sweep(4)
    assert np.array_equal(a.get_links(), b.get_links())
    a.close()
    b.close()


def test_library_allocated_memory_path():
    dims = (4, 4, 4, 4)
    a = Lattice(dims, 2.1, seed=4, start="hot", prec="f64", torch_memory=False)
    b = Lattice(dims, 2.1, seed=4, start="hot", prec="f64")
    a.sweep(2)
    b.sweep(2)
    assert np.array_equal(a.get_links(), b.get_links())
    a.close()
    b.close()


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_batched_sweep_parity(prec):
    dims = [(4, 4, 4, 4), (6, 4, 4, 2), (2, 4, 6, 4), (8, 8, 8, 8)]
    betas = [2.0, 2.5, 0.0, 2.7]
    b = Batch(dims, betas, seed=13, start="hot", prec=prec)
    nsw = 2 if prec == "f64" else 1
    b.sweep(nsw)
    for i, d in enumerate(dims):
        ch = oracle.chain(betas[i], seed=13, lattice_id=i, u23=u23(prec))
        U = oracle.init_hot(list(d), ch)
        for sw in range(nsw):
            oracle.sweep(list(d), U, ch, sw)
        diff = np.abs(b.get_links(i) - U).max(axis=-1)
        if prec == "f64":
            assert diff.max() < 1e-12, (i, diff.max())
        else:
            # FP32 after a full sweep: a decision that rounding flips changes
            # that link and, through the staples, a few later ones; all other
            # links agree to FP32 accuracy.
            assert (diff < TOL[prec]).mean() > 0.99, (i, (diff >= TOL[prec]).sum())
    plq = b.plaquette()
    pol = b.polyakov()
    for i, d in enumerate(dims):
        U = b.get_links(i)
        np.testing.assert_allclose(plq[i], oracle.plaquette(list(d), U), atol=MTOL[prec], rtol=0)
        assert abs(pol[i] - oracle.polyakov(list(d), U)) < MTOL[prec]
    b.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "f16q"])
def test_batched_measured_sweeps_against_the_oracle(prec):
    # every sweep's plaquette and Polyakov loop of every lattice against the
    # oracle's measurements of the same links (a twin batch swept one sweep
    # at a time; the chain itself is compared with the oracle in
    # test_batched_sweep_parity), with one group per lattice and with one
    # group for all; the 16^3 x 8 lattice's group spans many CTAs
    dims = [(4, 4, 4, 4), (6, 4, 4, 2), (16, 16, 16, 8), (2, 4, 6, 4)]
    betas = [2.0, 2.5, 2.3, 0.0]
    b = Batch(dims, betas, seed=17, start="hot", prec=prec)
    twin = Batch(dims, betas, seed=17, start="hot", prec=prec)
    for G in (len(dims), 1):
        b.groups = G
        hist = b.sweep_measure(3)
        assert hist.shape == (3, len(dims), 4)
        for sw in range(3):
            twin.sweep(1)
            for i, d in enumerate(dims):
                U = twin.get_links(i)
                ref = list(oracle.plaquette(list(d), U)) + [oracle.polyakov(list(d), U)]
                np.testing.assert_allclose(hist[sw, i], ref, atol=MTOL[prec], rtol=0)
        for i in range(len(dims)):
            assert np.array_equal(b.get_links(i), twin.get_links(i))   # measuring leaves the chain alone
    b.close()
    twin.close()


@pytest.mark.parametrize("dims,start", [([(8, 8, 8, 8), (4, 4, 4, 8)], "hot"), ([(8, 8, 8, 8)], "cold")])
def test_batched_measured_sweep_matches_the_single_lattice_history(dims, start):
    # lattice i of a batch is the single-lattice chain with lattice_id i; for
    # lattice 0 (lattice_id 0) the batched history equals su2_sweep_measure's
    # (a batch of one small lattice runs on a few CTAs only)
    b = Batch(dims, [2.4, 2.2][:len(dims)], seed=5, start=start, prec="f64")
    hist = b.sweep_measure(4)
    lat = Lattice(dims[0], 2.4, seed=5, start=start, prec="f64")
    ref = lat.sweep_measure(4)
    np.testing.assert_allclose(hist[:, 0, :], ref, atol=1e-12, rtol=0)
    lat.close()
    b.close()


def test_batched_rejects_a_member_beyond_32_bit_offsets():
    # 512^3 x 8 = 2^30 sites (a valid single lattice): the batched kernel's
    # 32-bit link offsets do not reach it; rejected before anything is allocated
    with pytest.raises(SU2Error, match="2\\^30"):
        Batch([(8, 8, 8, 8), (512, 512, 512, 8)], [2.3, 2.3], seed=1, prec="f32")


def test_batched_result_is_independent_of_the_schedule():
    dims = [(4, 4, 4, 4), (6, 4, 4, 2), (8, 8, 8, 8), (6, 6, 6, 4), (4, 4, 2, 8)]
    betas = [2.0, 2.5, 2.7, 0.0, 2.2]
    ref = None
    for G, bs in ((1, 256), (2, 512), (3, 256), (5, 512)):
        b = Batch(dims, betas, seed=31, start="hot", prec="f32")
        b.block_size = bs
        b.groups = G
        assert b.groups == G and b.block_size == bs
        b.sweep(3)
        links = [b.get_links(i) for i in range(len(dims))]
        b.close()
        if ref is None:
            ref = links
        else:
            for a, c in zip(ref, links):
                assert np.array_equal(a, c)


def test_batched_tuner_keeps_the_chain():
    dims = [(8, 8, 8, 8), (6, 6, 6, 6), (4, 4, 4, 4)]
    a = Batch(dims, [2.3, 2.4, 2.5], seed=41, start="hot", prec="f32")
    b = Batch(dims, [2.3, 2.4, 2.5], seed=41, start="hot", prec="f32")
    g = a.tune(2)
    assert 1 <= g <= 3 and a.groups == g
    a.sweep(2)
    b.sweep(2)
    for i in range(3):
        assert np.array_equal(a.get_links(i), b.get_links(i))
    with pytest.raises(SU2Error):
        a.groups = 4
    a.close()
    b.close()


def test_batched_tuning_cache(tmp_path):
    # the first tune times the candidates and records the winner under (GPU,
    # precision, shapes); a batch of the same shapes (other couplings, other
    # order) takes it from the cache without timing
    path = str(tmp_path / "tune.json")
    dims = [(8, 8, 8, 8), (6, 6, 6, 6), (4, 4, 4, 4), (8, 8, 8, 8)]
    a = Batch(dims, [2.3, 2.4, 2.5, 2.2], seed=41, start="hot", prec="f32")
    g = a.tune(2, cache=path)
    from paper_1010_4834_gb300 import tuning
    bs = a.block_size
    a.close()
    assert bs in (256, 512)
    assert list(tuning.load(path).values()) == [{"groups": g, "block_size": bs, "sweeps_timed": 2}]
    b = Batch(dims[::-1], [2.0, 2.1, 2.6, 2.7], seed=5, start="hot", prec="f32")
    assert b.tune(2, cache=path) == g and b.groups == g and b.block_size == bs
    b.close()


def test_batched_matches_single_lattice_chain():
    dims = [(4, 4, 4, 4), (6, 6, 6, 4)]
    b = Batch(dims, [2.2, 2.6], seed=21, start="hot", prec="f64")
    b.sweep(3)
    for i, d in enumerate(dims):
        ch = oracle.chain([2.2, 2.6][i], seed=21, lattice_id=i)
        U = oracle.init_hot(list(d), ch)
        for sw in range(3):
            oracle.sweep(list(d), U, ch, sw)
        assert np.abs(b.get_links(i) - U).max() < 1e-12
    b.close()


def test_batched_handle_recovers_after_a_timeout():
    """SU2_FAULT=barrier_once injects the missing arrival into the first
    batched sweep only.  That call reports SU2_ETIMEOUT and leaves the sweep
    counter where it was; after the links are reloaded the next sweep runs
    the oracle's sweep 0 from them, link for link."""
    dims = [(4, 4, 4, 4), (6, 4, 4, 2)]
    betas = [2.2, 2.5]
    os.environ["SU2_FAULT"] = "barrier_once"
    try:
        b = Batch(dims, betas, seed=17, start="hot", prec="f64")
    finally:
        del os.environ["SU2_FAULT"]
    with pytest.raises(SU2Error) as e:
        b.sweep(1)
    assert e.value.code == 4
    start = []
    for i, d in enumerate(dims):
        start.append(inputs.random_field(d, 60 + i))
        b.set_links(i, start[i])
    b.sweep(1)
    for i, d in enumerate(dims):
        ch = oracle.chain(betas[i], seed=17, lattice_id=i)
        U = start[i].copy()
        oracle.sweep(list(d), U, ch, 0)
        assert np.abs(b.get_links(i) - U).max() < 1e-12
    b.close()


def test_batched_barrier_timeout_is_reported():
    """Fault injection on the host side: the barrier waits for one arrival
    that never comes; every bounded wait runs out and the call reports
    SU2_ETIMEOUT without hanging or faulting, and the GPU stays usable."""
    os.environ["SU2_FAULT"] = "barrier"
    try:
        b = Batch([(4, 4, 4, 4)], [2.0], seed=1, start="cold", prec="f32")
    finally:
        del os.environ["SU2_FAULT"]
    with pytest.raises(SU2Error) as e:
        b.sweep(1)
    assert e.value.code == 4
    b.close()
    lat = Lattice((4, 4, 4, 4), 2.0, prec="f32")
    lat.sweep(1)
    assert lat.plaquette()[0] < 1.0
    lat.close()


# ---------------------------------------------------------------------------
def test_full_size_64_wilson_loops():
    """W(16,16) on 64^4 FP32 in the benchmark's launch configuration (the
    temporal-gauge kernel with eight origin rows a lane) against the FP64
    time-outer kernel, which is pinned to the oracle, on the same links."""
    dims = (64, 64, 64, 64)
    a = Lattice(dims, 2.6, seed=1, start="hot", prec="f32")
    a.sweep(2)
    U = a.get_links()
    w32 = a.wilson_loops(16, 16)
    a.close()
    b = Lattice(dims, 2.6, prec="f64")
    b.set_links(U)
    w64 = b.wilson_loops(16, 16)
    b.close()
    np.testing.assert_allclose(w32, w64, atol=1e-6, rtol=0)


def test_full_size_64_sampled():
    """64^4 FP32 (the benchmark's lattice and launch configuration): hot start,
    one heat-bath substep and the plaquette, checked on sampled links."""
    dims = (64, 64, 64, 64)
    beta = 2.6
    lat = Lattice(dims, beta, seed=1, start="hot", prec="f32")
    U0 = lat.get_links()
    ch = oracle.chain(beta, seed=1, u23=1)
    rng = np.random.default_rng(0)
    V = 64 ** 4
    for s in rng.integers(0, V, 300):
        for mu in range(4):
            assert np.abs(U0[s, mu] - oracle.hot_link(ch, s, mu)).max() < 2e-6
    lat.substep(1, 1, 0)
    U1 = lat.get_links()
    x = lambda s: (s % 64 + s // 64 % 64 + s // 4096 % 64 + s // 262144) % 2
    checked = 0
    for s in rng.integers(0, V, 4000):
        s = int(s)
        if x(s) != 1:
            assert np.array_equal(U1[s], U0[s])
            continue
        assert np.array_equal(U1[s, [0, 2, 3]], U0[s, [0, 2, 3]])
        sig = oracle.staple(list(dims), U0, s, 1)
        n, new, m = oracle.heatbath_link(ch, s, 1, 0, sig, U0[s, 1])
        if m < 1e-4:
            continue
        assert np.abs(U1[s, 1] - new).max() < 2e-5, (s, U1[s, 1], new)
        checked += 1
    assert checked > 1500
    p = lat.plaquette()
    assert abs(p[0] - oracle.plaquette(list(dims), U1)[0]) < 2e-7
    lat.close()


@pytest.mark.parametrize("beta,max_tries,schedule", [(2.6, 64, "pair"), (0.05, 64, "pair"), (2.6, 1, "pair"),
                                                     (2.6, 64, "substep"), (0.05, 64, "substep")])
def test_full_size_64_measured_sweep_every_substep_class(beta, max_tries, schedule):
    """64^4 FP32, the benchmark's lattice, in both sweep schedules: the fused
    parity pairs (the default there) and the substeps, which run 1024-thread
    blocks sharing one deferral queue.  One measured sweep (sweep_measure,
    whose parity-1 halves of mu = 1, 2, 3 are the plaquette-summing variant)
    from the hot start; every one of the eight (mu, parity) classes is checked on sampled
    links against the oracle's heat-bath draw from the state that substep saw
    (classes before it final, the others still at the start).  beta = 0.05
    makes most first trials fail (queue overflow, links finished inline,
    trials exhausted); max_tries = 1 keeps every rejected link.  The
    sweep's plaquette and Polyakov loop are compared with the oracle's on the
    final links."""
    dims = (64, 64, 64, 64)
    V = 64 ** 4
    lat = Lattice(dims, beta, seed=3, start="hot", prec="f32")
    lat.set_options(max_tries, "kp")
    lat.set_schedule(schedule)
    U0 = lat.get_links()
    hist = lat.sweep_measure(1)
    U1 = lat.get_links()
    lat.close()
    ch = oracle.chain(beta, seed=3, max_tries=max_tries, u23=1)
    s_all = np.arange(V)
    par = (s_all % 64 + s_all // 64 % 64 + s_all // 4096 % 64 + s_all // 262144) & 1
    rng = np.random.default_rng(int(beta * 100) + max_tries)
    comp = U0.copy()           # the state the next substep sees
    checked = kept = 0
    for mu in range(4):
        for p in range(2):
            sites = rng.choice(np.flatnonzero(par == p), 600, replace=False)
            for s in sites:
                s = int(s)
                sig = oracle.staple(list(dims), comp, s, mu)
                n, new, m = oracle.heatbath_link(ch, s, mu, 0, sig, comp[s, mu])
                if m < 1e-4:
                    continue
                assert np.abs(U1[s, mu] - new).max() < 2e-5, (mu, p, s, n, U1[s, mu], new)
                checked += 1
                kept += n == 0
            comp[par == p, mu] = U1[par == p, mu]
    assert checked > 8 * 450, checked
    if max_tries == 1 or beta < 0.1:
        assert kept > 0
    ref_p = oracle.plaquette(list(dims), U1)
    # FP32 per-thread sums of ~55 terms per thread, FP64 above that: a few
    # 1e-8 relative; the bar leaves room for the links' own FP32 rounding
    np.testing.assert_allclose(hist[0, :3], ref_p, rtol=0, atol=1e-6)
    assert abs(hist[0, 3] - oracle.polyakov(list(dims), U1)) < 1e-6


# ---------------------------------------------------------------------------
def test_sweep_measure_restart_and_launch_count():
    from paper_1010_4834_gb300 import kernel_launches
    dims = (4, 4, 6, 4)
    a = Lattice(dims, 2.3, seed=5, start="hot", prec="f64")
    b = Lattice(dims, 2.3, seed=5, start="hot", prec="f64")
    n0 = kernel_launches()
    hist = a.sweep_measure(6)
    assert kernel_launches() - n0 == 6 * (8 + 1)      # 8 substeps, Polyakov (+ plaquette, counter)
    ref = []
    for _ in range(6):
        b.sweep(1)
        ref.append(list(b.plaquette()) + [b.polyakov()])
    ref = np.array(ref)
    # the plaquette comes from the sweep's own staples: same sum, other order
    np.testing.assert_allclose(hist[:, :3], ref[:, :3], rtol=0, atol=1e-14)
    np.testing.assert_array_equal(hist[:, 3], ref[:, 3])
    np.testing.assert_array_equal(a.get_links(), b.get_links())
    assert a.sweep_count == 6
    a.restart("hot")
    assert a.sweep_count == 0
    fresh = Lattice(dims, 2.3, seed=5, start="hot", prec="f64")
    assert np.array_equal(a.get_links(), fresh.get_links())
    for lat in (a, b, fresh):
        lat.close()


# Runs of 8 measured sweeps replay as a graph and write a history ring indexed
# by the sweep counter: a run that starts 4 rows before the ring's end, wraps
# and spans two host chunks (1024 rows each) must match sweep-by-sweep
# measurements row for row, and leave the same links and counter.
def test_sweep_measure_graph_ring_wrap_and_chunks():
    from paper_1010_4834_gb300 import kernel_launches
    dims = (4, 4, 4, 6)
    a = Lattice(dims, 2.3, seed=9, start="hot", prec="f64")
    b = Lattice(dims, 2.3, seed=9, start="hot", prec="f64")
    a.sweep_count = 1020
    b.sweep_count = 1020
    n = 1030
    n0 = kernel_launches()
    hist = a.sweep_measure(n)
    assert kernel_launches() - n0 == 9 * n
    assert hist.shape == (n, 4)
    rows = [0, 1, 3, 4, 5, 11, 12, 1023, 1024, 1025, n - 1]
    ref = {}
    for i in range(n):
        b.sweep(1)
        if i in rows:
            ref[i] = list(b.plaquette()) + [b.polyakov()]
    for i in rows:
        np.testing.assert_allclose(hist[i, :3], ref[i][:3], rtol=0, atol=1e-14, err_msg="row %d" % i)
        assert hist[i, 3] == ref[i][3], i
    assert len(np.unique(hist[:, 3])) > n // 2      # every row was written
    np.testing.assert_array_equal(a.get_links(), b.get_links())
    assert a.sweep_count == b.sweep_count == 1020 + n
    for lat in (a, b):
        lat.close()


# The plaquette that sweep_measure takes from the odd-parity substeps of
# mu = 1, 2, 3 against the plaquette kernel run after a plain sweep: every
# branch of the update (first-trial accept, deferred trials, capped link
# kept, Haar link at beta = 0, Creutz; the queue overflow is covered on 48^4
# below), each precision, a lattice of several blocks with a ragged last one.  The measured sweeps must leave the
# same links as plain ones.
@pytest.mark.parametrize("prec,tol", [("f64", 1e-14), ("f32", 3e-6), ("f16q", 3e-6)])
@pytest.mark.parametrize("beta,max_tries,sampler", [
    (2.3, 64, "kp"),      # mostly first-trial accepts, a few deferred
    (0.4, 64, "kp"),      # low acceptance: many deferred
    (2.3, 1, "kp"),       # capped links keep their old value
    (0.0, 64, "kp"),      # alpha = 0: Haar links
    (2.3, 64, "creutz"),
])
def test_sweep_plaquette_matches_plaquette_kernel(prec, tol, beta, max_tries, sampler):
    dims = (8, 6, 4, 10)                 # V/2 = 960: four blocks, the last one partial
    a = Lattice(dims, beta, seed=41, start="hot", prec=prec)
    b = Lattice(dims, beta, seed=41, start="hot", prec=prec)
    for lat in (a, b):
        lat.set_options(max_tries=max_tries, sampler=sampler)
    hist = a.sweep_measure(3)
    for i in range(3):
        b.sweep(1)
        np.testing.assert_allclose(hist[i, :3], b.plaquette(), rtol=0, atol=tol)
        assert hist[i, 3] == b.polyakov()
    np.testing.assert_array_equal(a.get_links(), b.get_links())
    a.close()
    b.close()


@pytest.mark.parametrize("n,beta", [(32, 2.5), (48, 0.05)])
def test_sweep_plaquette_full_size_grid(n, beta):
    # the substeps run the full persistent grid, several iterations per block;
    # at beta 0.05 on 48^4 (17 iterations of 1024 links per block) most first
    # trials fail, the block queues overflow (4096 entries) and some links
    # exhaust their trials
    a = Lattice((n,) * 4, beta, seed=43, start="hot", prec="f32")
    b = Lattice((n,) * 4, beta, seed=43, start="hot", prec="f32")
    hist = a.sweep_measure(2)
    b.sweep(2)
    np.testing.assert_allclose(hist[-1, :3], b.plaquette(), rtol=0, atol=2e-6)
    np.testing.assert_array_equal(a.get_links(), b.get_links())
    a.close()
    b.close()


@pytest.mark.parametrize("dims,max_tries", [((8, 6, 4, 10), 64), ((16, 16, 16, 16), 64), ((8, 8, 8, 8), 1)])
def test_layout_comparison_runs_the_same_chain(dims, max_tries):
    # Section 5.1's one-array layout and the plain kernel on the library's
    # layout leave the same links as the library's kernels; the handle keeps
    # that result and the counter advances
    a = Lattice(dims, 2.4, seed=9, start="hot", prec="f32")
    b = Lattice(dims, 2.4, seed=9, start="hot", prec="f32")
    for lat in (a, b):
        lat.set_options(max_tries=max_tries)
    ms, mismatch = a.layout_compare(3)
    assert mismatch == 0
    assert np.all(ms > 0)
    b.sweep(3)
    np.testing.assert_array_equal(a.get_links(), b.get_links())
    assert a.sweep_count == 3
    with pytest.raises(SU2Error):
        a.layout_compare(0)
    c = Lattice((4, 4, 4, 4), 2.0, prec="f64")
    with pytest.raises(SU2Error):
        c.layout_compare(1)
    for lat in (a, b, c):
        lat.close()


def test_work_is_ordered_on_the_torch_stream():
    import torch
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        lat = Lattice((8, 8, 8, 8), 2.4, seed=3, start="hot", prec="f32")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        lat.sweep(16)
        e1.record()
        e1.synchronize()
        # the events bracket the sweeps: a 16-sweep run takes measurable time
        assert e0.elapsed_time(e1) > 0.005
        assert lat.sweep_count == 16
        lat.close()
