"""Static quark-antiquark potential from Wilson loops (Section 5.4).

Host-side analysis of the W(R, T) that su2_wilson_loops returns:
  * effective potential V(R) = ln(W(R,T) / W(R,T+1)) (Eq. 23), which tends to
    the ground-state energy as T grows because <W(R,T)> ~ exp(-T V(R)) (Eq. 24);
  * the fit a V(a R) = A a + B / R + sigma a^2 R (Eq. 22), by weighted linear
    least squares in the three parameters;
  * the lattice spacing a = sqrt(sigma a^2) * 197 MeV fm / 440 MeV (Eq. 25,
    with the physical string tension sqrt(sigma) = 440 MeV).
"""
import numpy as np

HBARC_MEV_FM = 197.0
SQRT_SIGMA_MEV = 440.0


def effective_potential(W):
    """V[R-1, T-1] = ln(W(R,T) / W(R,T+1)) for a W[R-1, T-1] array; shape (Rmax, Tmax-1)."""
    W = np.asarray(W, float)
    return np.log(W[:, :-1] / W[:, 1:])


def fit_potential(R, V, err=None):
    """Fit V(R) = A + B/R + s R.  Returns (A, B, s) and their covariance."""
    R = np.asarray(R, float)
    V = np.asarray(V, float)
    w = np.ones_like(V) if err is None else 1.0 / np.asarray(err, float) ** 2
    X = np.stack([np.ones_like(R), 1.0 / R, R], axis=1)
    XtW = X.T * w
    cov = np.linalg.inv(XtW @ X)
    coef = cov @ (XtW @ V)
    return coef, cov


def lattice_spacing_fm(sigma_a2):
    """a in fm from the fitted string tension in lattice units (Eq. 25)."""
    return np.sqrt(np.asarray(sigma_a2, float)) * HBARC_MEV_FM / SQRT_SIGMA_MEV


# ---------------------------------------------------------------------------
# From an ensemble of configurations
# ---------------------------------------------------------------------------
def wilson_ensemble(lat, nconf, every, alpha=0.7, n_ape=25, rmax=8, tmax=8):
    """W(R,T) of `nconf` configurations of the chain `lat` (a Lattice), taken
    `every` heat-bath sweeps apart, each after `n_ape` APE steps (Eq. 19) of
    its spatial links; shape (nconf, rmax, tmax).  All of it runs in the
    library's kernels; this loop only collects the results."""
    out = np.empty((nconf, rmax, tmax))
    for i in range(nconf):
        lat.sweep(every)
        lat.ape_smear(alpha, n_ape)
        out[i] = lat.wilson_loops(rmax, tmax, smeared=True)
    return out


def jackknife(samples, fn):
    """Delete-one jackknife of fn applied to the mean over the first axis:
    (fn of the full mean, error, fn of each delete-one mean)."""
    samples = np.asarray(samples, float)
    n = len(samples)
    tot = samples.sum(axis=0)
    full = fn(tot / n)
    reps = np.array([fn((tot - samples[i]) / (n - 1)) for i in range(n)])
    err = np.sqrt((n - 1) / n * ((reps - reps.mean(axis=0)) ** 2).sum(axis=0))
    return full, err, reps


def _veff(W):
    with np.errstate(divide="ignore", invalid="ignore"):
        return effective_potential(W)


def static_potential(W_samples, rfit=None, nsig=1.5, tmin=2):
    """Static potential from W(R,T) samples (nconf, Rmax, Tmax).

    V(R,T) = ln(W(R,T)/W(R,T+1)) (Eq. 23) with jackknife errors.  For every R
    the plateau is the first T >= tmin at which V(R,T) and V(R,T+1) agree
    within `nsig` jackknife errors of their difference (excited states have
    decayed, Eq. 24; T = 1 is left out by default, since loops one slice long
    still carry the contact terms); V(R) is V(R, T_plateau).  Then A + B/R + sigma R (Eq. 22) is
    fitted over R = 1..rfit (default: every R with a finite plateau value),
    weighted by the errors of V(R), with jackknife errors of the parameters,
    and the lattice spacing follows from sigma (Eq. 25)."""
    W_samples = np.asarray(W_samples, float)
    rmax, tmax = W_samples.shape[1:]
    Vt, dVt, _ = jackknife(W_samples, _veff)                       # (rmax, tmax - 1)
    _, ddiff, _ = jackknife(W_samples, lambda w: np.diff(_veff(w), axis=1))
    tp = np.full(rmax, tmax - 1)
    for r in range(rmax):
        for t in range(tmin - 1, tmax - 2):
            d = Vt[r, t] - Vt[r, t + 1]
            if np.isfinite(d) and abs(d) <= nsig * ddiff[r, t]:
                tp[r] = t + 1
                break
    rows = np.arange(rmax)
    V, dV, Vreps = jackknife(W_samples, lambda w: _veff(w)[rows, tp - 1])
    ok = np.isfinite(V) & np.isfinite(dV) & (dV > 0)
    nfit = rfit if rfit is not None else int(np.argmin(ok)) if not ok.all() else rmax
    R = np.arange(1, nfit + 1)
    err = dV[:nfit]
    coef, _ = fit_potential(R, V[:nfit], err)
    rep_coef = np.array([fit_potential(R, v[:nfit], err)[0] for v in Vreps])
    n = len(W_samples)
    cerr = np.sqrt((n - 1) / n * ((rep_coef - rep_coef.mean(axis=0)) ** 2).sum(axis=0))
    sigma, dsigma = float(coef[2]), float(cerr[2])
    a = float(lattice_spacing_fm(sigma)) if sigma > 0 else float("nan")
    return {"V_RT": Vt, "dV_RT": dVt, "T_plateau": tp, "V": V, "dV": dV, "rfit": nfit,
            "coef": coef, "coef_err": cerr, "sigma_a2": sigma, "sigma_a2_err": dsigma,
            "a_fm": a, "a_fm_err": a * 0.5 * dsigma / sigma if sigma > 0 else float("nan")}
