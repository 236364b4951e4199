"""Ensemble parity: FP32, F16Q and batched chains against the FP64 chain.

Past the first sweep the chains of different precisions separate (a rounding
difference flips an accept decision, after which the trajectories are
unrelated), so they are compared as Monte Carlo ensembles: means of the
plaquette, |Polyakov loop| and small Wilson loops over many sweeps, with
errors from binning (bins long against the autocorrelation time), must agree
within 3 combined standard deviations.  The FP64 chain itself agrees with the
oracle link by link (test_gpu_parity.py).  Chains use different seeds, so
they are statistically independent.
"""
import numpy as np
import pytest

from paper_1010_4834_gb300 import Batch, Lattice

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.set_device(0)


def binned(x, nbins=40):
    x = np.asarray(x, float)
    x = x[: len(x) // nbins * nbins].reshape(nbins, -1).mean(1)
    return x.mean(), x.std(ddof=1) / np.sqrt(nbins)


def agree(a, b, nsig=3.0):
    (ma, ea), (mb, eb) = a, b
    return abs(ma - mb) <= nsig * np.hypot(ea, eb), (ma, ea, mb, eb)


def chain_history(dims, beta, prec, seed, ntherm, nmeas):
    lat = Lattice(dims, beta, seed=seed, start="hot", prec=prec)
    lat.sweep(ntherm)
    h = lat.sweep_measure(nmeas)
    lat.close()
    return h


@pytest.fixture(scope="module")
def ref_8x4():
    return chain_history((8, 8, 8, 8), 2.4, "f64", 101, 200, 4000)


@pytest.mark.parametrize("prec", ["f32", "f16q"])
def test_plaquette_ensemble(ref_8x4, prec):
    h = chain_history((8, 8, 8, 8), 2.4, prec, 202, 200, 4000)
    for k in range(3):                          # all, spatial, space-time
        ok, info = agree(binned(h[:, k]), binned(ref_8x4[:, k]))
        assert ok, (prec, k, info)


@pytest.mark.parametrize("prec", ["f32", "f16q"])
def test_polyakov_modulus_ensemble_finite_temperature(prec):
    # 8^3 x 4 at beta 2.5 is above the Nt = 4 deconfinement coupling: |L| > 0
    ref = chain_history((8, 8, 8, 4), 2.5, "f64", 303, 300, 4000)
    h = chain_history((8, 8, 8, 4), 2.5, prec, 404, 300, 4000)
    a, b = binned(np.abs(h[:, 3])), binned(np.abs(ref[:, 3]))
    assert a[0] > 0.1
    ok, info = agree(a, b)
    assert ok, (prec, info)
    ok, info = agree(binned(h[:, 0]), binned(ref[:, 0]))
    assert ok, (prec, info)


def wilson_history(prec, seed, n=600, every=4):
    lat = Lattice((8, 8, 8, 8), 2.3, seed=seed, start="hot", prec=prec)
    lat.sweep(200)
    out = []
    for _ in range(n):
        lat.sweep(every)
        lat.ape_smear(0.5, 2)
        out.append(lat.wilson_loops(3, 3, smeared=True).ravel())
    lat.close()
    return np.array(out)


def test_smeared_wilson_loop_ensemble_fp32():
    ref = wilson_history("f64", 505)
    got = wilson_history("f32", 606)
    for j in range(ref.shape[1]):
        ok, info = agree(binned(got[:, j], 30), binned(ref[:, j], 30))
        assert ok, (j, info)


def test_batched_ensemble_against_single_lattices():
    dims = [(8, 8, 8, 8), (6, 6, 6, 6)]
    betas = [2.4, 2.2]
    b = Batch(dims * 4, betas * 4, seed=707, start="hot", prec="f32")
    b.sweep(200)
    plq = []
    for _ in range(1000):
        b.sweep(2)
        plq.append(b.plaquette()[:, 0])
    b.close()
    plq = np.array(plq)                        # (sweeps, 8 lattices)
    for i, (d, be) in enumerate(zip(dims, betas)):
        mine = plq[:, i::2].mean(axis=1)       # the four copies of this shape, averaged
        ref = chain_history(d, be, "f64", 808 + i, 200, 2000)[:, 0]
        ok, info = agree(binned(mine), binned(ref))
        assert ok, (d, info)


def test_finite_temperature_scan_reduced_precisions_match_fp64():
    """The 32^3 x 4 scan at 16 couplings in [2.2, 2.6] (cold start, 1000
    sweeps each, the first 300 dropped): FP32 and F16Q plaquette and |Polyakov loop| against
    the FP64 ensemble at every coupling.  With 64 comparisons a 3-sigma cut
    would fail by chance about one run in six, so each deviation must stay
    within 4 combined errors and their mean square near 1; and |L| must show
    the transition (small at 2.2, large at 2.6)."""
    from paper_1010_4834_gb300.ensemble import deviation, scan
    res = scan()
    z = []
    for k, (beta, p64, l64) in enumerate(res["f64"]):
        for prec in ("f32", "f16q"):
            _, p, l = res[prec][k]
            z += [deviation(p, p64), deviation(l, l64)]
    z = np.array(z)
    assert np.all(np.abs(z) < 4), z
    assert np.mean(z ** 2) < 2.0, np.mean(z ** 2)
    l_lo, l_hi = res["f64"][0][2][0], res["f64"][-1][2][0]
    assert l_lo < 0.1 < 0.2 < l_hi, (l_lo, l_hi)
