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
