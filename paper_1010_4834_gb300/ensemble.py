"""Monte Carlo ensembles and their statistics: the plaquette (Section 5.2)
and the Polyakov loop as a function of beta (Section 5.3, the order
parameter of the deconfinement transition at finite temperature, Eqs. 14-15).

A chain is a lattice swept with su2_sweep_measure, which records the
plaquette and the Polyakov loop after every sweep; the first 20% of the
sweeps are discarded as thermalisation.  Errors come from binning: the
series is cut into bins of 2^k consecutive sweeps, k = 0, 1, 2, ..., and the
error of the mean is the spread of the bin means over sqrt(number of bins).
For an autocorrelated series that error grows with the bin size until the
bins are long against the autocorrelation time, then stays flat; the first
bin size from which it stays flat (within the statistical uncertainty of an
error estimate from that many bins) is the plateau, and its error is the
one quoted.  Two ensembles agree at n sigma when their means differ by less
than n combined errors.

Run as a module on a GPU to print the scan of the 32^3 x 4 lattice at 16
couplings in [2.2, 2.6] for FP64, FP32 and F16Q storage, with each reduced
precision's deviation from the FP64 ensemble in units of the combined error:

    python -m paper_1010_4834_gb300.ensemble [sweeps]
"""
import sys
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .lattice import Batch, Lattice

THERM_FRACTION = 0.2
MIN_BINS = 16


def binned(x, nbins=20):
    """Mean and binned error of a series with a fixed bin count (the tail
    that does not fill a bin is dropped)."""
    x = np.asarray(x, float)
    m = len(x) // nbins * nbins
    b = x[:m].reshape(nbins, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / np.sqrt(nbins))


def binning_curve(x, min_bins=MIN_BINS):
    """[(bin size 2^k, error of the mean, number of bins)] for every k that
    leaves at least `min_bins` bins."""
    x = np.asarray(x, float)
    out = []
    b = 1
    while len(x) // b >= min_bins:
        nb = len(x) // b
        m = x[: nb * b].reshape(nb, b).mean(axis=1)
        out.append((b, float(m.std(ddof=1) / np.sqrt(nb)), nb))
        b *= 2
    return out


def plateau_binned(x, min_bins=MIN_BINS):
    """Mean of x and its error at the binning plateau.

    Returns (mean, error, bin size, plateau reached).  The plateau is the
    smallest bin size b_k whose error e_k no later bin size exceeds by more
    than twice the relative uncertainty 1/sqrt(2 (n_j - 1)) of an error
    estimated from n_j bins; the error quoted is the mean of the errors from
    b_k on (they estimate the same number).  If the error is still growing
    at the largest bin size that leaves `min_bins` bins, the series is too
    short for its autocorrelation: the largest error is returned with
    plateau reached = False."""
    x = np.asarray(x, float)
    curve = binning_curve(x, min_bins)
    if not curve:
        raise ValueError("series of %d values is too short for %d bins" % (len(x), min_bins))
    errs = np.array([e for _, e, _ in curve])
    rel = np.array([1.0 / np.sqrt(2.0 * (nb - 1)) for _, _, nb in curve])
    for k in range(len(curve)):
        if np.all(errs[k + 1:] <= errs[k] * (1.0 + 2.0 * rel[k + 1:])):
            # a plateau needs at least one larger bin size to confirm it
            if k + 1 < len(curve):
                return float(x.mean()), float(errs[k:].mean()), curve[k][0], True
            break
    return float(x.mean()), float(errs.max()), curve[int(np.argmax(errs))][0], False


def deviation(a, b):
    """(mean_a - mean_b) / combined error for two (mean, error[, ...]) tuples."""
    ma, ea = a[0], a[1]
    mb, eb = b[0], b[1]
    return (ma - mb) / float(np.hypot(ea, eb))


def thermalised(h, frac=THERM_FRACTION):
    """The series with its first `frac` dropped as thermalisation."""
    return h[int(round(frac * len(h))):]


def chain(dims, beta, prec, seed, sweeps, start="cold"):
    """History (sweeps, 4) of plaquette (all, spatial, space-time) and
    Polyakov loop after each measured sweep, thermalisation included."""
    lat = Lattice(dims, beta, seed=seed, start=start, prec=prec)
    h = lat.sweep_measure(sweeps)
    lat.close()
    return h


def chains(specs, sweeps, start="cold", workers=8, overrelax=0):
    """Many independent single-lattice chains at once: specs is a list of
    (dims, beta, prec, seed).  Each chain runs on its own CUDA stream from its
    own host thread (a small lattice fills only part of the GPU), with
    `overrelax` over-relaxation sweeps before every measured heat-bath sweep.
    Returns the histories in the order of specs."""
    import torch

    dev = torch.cuda.current_device()

    def run(spec):
        torch.cuda.set_device(dev)
        dims, beta, prec, seed = spec
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            lat = Lattice(dims, beta, seed=seed, start=start, prec=prec, stream=s)
            if overrelax:
                lat.set_overrelax(overrelax)
            h = lat.sweep_measure(sweeps)
            lat.close()
        return h

    with ThreadPoolExecutor(max(1, min(workers, len(specs)))) as ex:
        return list(ex.map(run, specs))


def batch_chains(dims_list, betas, prec, seed, sweeps, start="cold", every=1, overrelax=0):
    """Histories of the lattices of one batched handle (su2_batch_*), all
    swept together (`overrelax` over-relaxation sweeps before every
    heat-bath sweep): (n, sweeps // every, 4) of plaquette (all, spatial,
    space-time) and Polyakov loop, measured every `every` sweeps."""
    b = Batch(dims_list, betas, seed=seed, start=start, prec=prec)
    if overrelax:
        b.set_overrelax(overrelax)
    n = len(dims_list)
    m = sweeps // every
    out = np.empty((n, m, 4))
    for i in range(m):
        b.sweep(every)
        out[:, i, :3] = b.plaquette()
        out[:, i, 3] = b.polyakov()
    b.close()
    return out


def observables(h):
    """The per-sweep series the ensembles are compared on: the plaquette and
    the modulus of the Polyakov loop, thermalisation dropped."""
    h = thermalised(h)
    return {"P": h[:, 0], "|L|": np.abs(h[:, 3])}


def compare(h, ref, nsig=3.0):
    """Plateau-binned means of each observable of history h and of the
    reference history, their deviation in combined errors and the plateau
    bin sizes: {name: dict}."""
    out = {}
    a, b = observables(h), observables(ref)
    for k in a:
        ma = plateau_binned(a[k])
        mb = plateau_binned(b[k])
        z = deviation(ma, mb)
        out[k] = {"mean": ma[0], "err": ma[1], "bin": ma[2], "plateau": ma[3],
                  "ref_mean": mb[0], "ref_err": mb[1], "ref_bin": mb[2], "ref_plateau": mb[3],
                  "dev": z, "ok": bool(abs(z) <= nsig)}
    return out


def scan(dims=(32, 32, 32, 4), betas=None, precs=("f64", "f32", "f16q"), sweeps=4000, seed=1, start="cold",
         overrelax=2):
    """For every coupling and precision: plateau-binned plaquette and
    |Polyakov loop| of chains of `sweeps` heat-bath sweeps, each preceded by
    `overrelax` over-relaxation sweeps (near the transition the Polyakov
    loop's autocorrelation time is hundreds of heat-bath sweeps).
    Returns {prec: [(beta, (P, dP, bin, ok), (L, dL, bin, ok)), ...]}.
    Each (beta, precision) chain has its own seed, so the ensembles are
    independent.  The default cold start matters above the transition: a hot
    start there freezes into domains of opposite Polyakov-loop sign whose
    interfaces outlive thousands of sweeps, which lowers |L| (and the
    plaquette) by amounts that differ from chain to chain; from the cold start
    the field stays in one sector."""
    if betas is None:
        betas = np.linspace(2.2, 2.6, 16)
    specs = [(dims, float(beta), prec, seed + 101 * i + 7 * j)
             for i, beta in enumerate(betas) for j, prec in enumerate(precs)]
    hs = chains(specs, sweeps, start=start, overrelax=overrelax)
    out = {p: [] for p in precs}
    for (d, beta, prec, _), h in zip(specs, hs):
        o = observables(h)
        out[prec].append((beta, plateau_binned(o["P"]), plateau_binned(o["|L|"])))
    return out


def main(sweeps=4000):
    res = scan(sweeps=sweeps)
    print("| beta | <P> FP64 | <P> FP32 (dev) | <P> F16Q (dev) | <|L|> FP64 | <|L|> FP32 (dev) | <|L|> F16Q (dev) "
          "| bins P / |L| (FP64) |")
    print("|---|---|---|---|---|---|---|---|")
    for k in range(len(res["f64"])):
        beta, p64, l64 = res["f64"][k]
        row = ["%.4f" % beta, "%.5f(%d)" % (p64[0], round(p64[1] * 1e5))]
        for prec in ("f32", "f16q"):
            p = res[prec][k][1]
            row.append("%.5f (%+.1f)" % (p[0], deviation(p, p64)))
        row.append("%.4f(%d)" % (l64[0], round(l64[1] * 1e4)))
        for prec in ("f32", "f16q"):
            l = res[prec][k][2]
            row.append("%.4f (%+.1f)" % (l[0], deviation(l, l64)))
        row.append("%d / %d" % (p64[2], l64[2]))
        print("| " + " | ".join(row) + " |")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 4000)
