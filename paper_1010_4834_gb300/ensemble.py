"""Monte Carlo ensembles and their statistics: the plaquette (Section 5.2)
and the Polyakov loop as a function of beta (Section 5.3, the order
parameter of the deconfinement transition at finite temperature, Eqs. 14-15).

A chain is a hot-started lattice swept with su2_sweep_measure, which records
the plaquette and the Polyakov loop after every sweep; the first sweeps are
discarded as thermalisation.  Errors come from binning: the measurements are
cut into a fixed number of consecutive bins, long against the
autocorrelation time, and the error of the mean is the spread of the bin
means over sqrt(number of bins).  Two ensembles agree when their means differ
by less than a few combined errors.

Run as a module on a GPU to print the scan of the 32^3 x 4 lattice at 16
couplings in [2.2, 2.6] for FP64, FP32 and F16Q storage, with each reduced
precision's deviation from the FP64 ensemble in units of the combined error:

    python -m paper_1010_4834_gb300.ensemble
"""
import numpy as np

from .lattice import Lattice


def binned(x, nbins=20):
    """Mean and binned error of a series (the tail that does not fill a bin is dropped)."""
    x = np.asarray(x, float)
    m = len(x) // nbins * nbins
    b = x[:m].reshape(nbins, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / np.sqrt(nbins))


def deviation(a, b):
    """(mean_a - mean_b) / combined error for two (mean, error) pairs."""
    (ma, ea), (mb, eb) = a, b
    return (ma - mb) / float(np.hypot(ea, eb))


def chain(dims, beta, prec, seed, sweeps, therm, start="hot"):
    """History (sweeps - therm, 4) of plaquette (all, spatial, space-time) and
    Polyakov loop after each measured sweep, thermalisation sweeps dropped."""
    lat = Lattice(dims, beta, seed=seed, start=start, prec=prec)
    h = lat.sweep_measure(sweeps)
    lat.close()
    return h[therm:]


def scan(dims=(32, 32, 32, 4), betas=None, precs=("f64", "f32", "f16q"), sweeps=1000, therm=300,
         seed=1, nbins=10, start="cold"):
    """For every coupling and precision: binned plaquette and |Polyakov loop|.
    Returns {prec: [(beta, (P, dP), (L, dL)), ...]}.  Each (beta, precision)
    chain has its own seed, so the ensembles are independent.  The default
    cold start matters above the transition: a hot start there freezes into
    domains of opposite Polyakov-loop sign whose interfaces outlive a
    thousand sweeps, which lowers |L| (and the plaquette) by amounts that
    differ from chain to chain; from the cold start the field stays in one
    sector."""
    if betas is None:
        betas = np.linspace(2.2, 2.6, 16)
    out = {p: [] for p in precs}
    for i, beta in enumerate(betas):
        for j, prec in enumerate(precs):
            h = chain(dims, float(beta), prec, seed + 101 * i + 7 * j, sweeps, therm, start)
            out[prec].append((float(beta), binned(h[:, 0], nbins), binned(np.abs(h[:, 3]), nbins)))
    return out


def main():
    res = scan()
    print("| beta | <P> FP64 | <P> FP32 (dev) | <P> F16Q (dev) | <|L|> FP64 | <|L|> FP32 (dev) | <|L|> F16Q (dev) |")
    print("|---|---|---|---|---|---|---|")
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
        print("| " + " | ".join(row) + " |")


if __name__ == "__main__":
    main()
