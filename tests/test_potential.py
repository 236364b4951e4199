"""Pins for the static-potential analysis (Section 5.4, Eqs. 22-25)."""
import os

import numpy as np

from paper_1010_4834_gb300 import potential

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lattice_spacing_table.txt")


def test_lattice_spacing_reproduces_the_paper_table():
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for beta, s, a, *_ in rows:
        # the table prints a(fm) to 6 decimals
        assert abs(potential.lattice_spacing_fm(float(s)) - float(a)) < 1.5e-6, (beta, s, a)


def test_effective_potential_and_fit_recover_a_known_potential():
    A, B, s = 0.55, -0.27, 0.041
    R = np.arange(1, 9)
    V = A + B / R + s * R
    T = np.arange(1, 11)
    c = 0.8 + 0.02 * R                      # overlaps of the trial state
    W = c[:, None] * np.exp(-np.outer(V, T))
    Veff = potential.effective_potential(W)
    assert Veff.shape == (8, 9)
    np.testing.assert_allclose(Veff, np.repeat(V[:, None], 9, axis=1), rtol=0, atol=1e-12)
    (fA, fB, fs), cov = potential.fit_potential(R, Veff[:, 3])
    np.testing.assert_allclose([fA, fB, fs], [A, B, s], atol=1e-10)
    # an excited state decays away with T: the plateau value is the ground state
    W2 = W + 0.3 * np.exp(-np.outer(V + 0.9, T))
    V2 = potential.effective_potential(W2)
    assert np.all(np.abs(V2[:, -1] - V) < np.abs(V2[:, 0] - V))


def test_weighted_fit_uses_the_errors():
    R = np.arange(1, 7).astype(float)
    V = 0.5 - 0.3 / R + 0.05 * R
    err = np.full_like(R, 1e-3)
    V_bad = V.copy()
    V_bad[-1] += 0.2
    err_bad = err.copy()
    err_bad[-1] = 1e3                        # the outlier carries no weight
    (a, b, s), _ = potential.fit_potential(R, V_bad, err_bad)
    np.testing.assert_allclose([a, b, s], [0.5, -0.3, 0.05], atol=1e-6)


def test_ensemble_analysis_recovers_the_string_tension():
    # synthetic ensemble: W(R,T) = c exp(-T V(R)) + excited state, with
    # independent noise per configuration; the plateau rule must skip the
    # small T where the excited state still shows, and the jackknife fit must
    # find sigma within its error
    A, B, s = 0.55, -0.27, 0.041
    R = np.arange(1, 8)
    T = np.arange(1, 9)
    V = A + B / R + s * R
    W = (0.9 * np.exp(-np.outer(V, T)) + 0.1 * np.exp(-np.outer(V + 0.8, T)))
    rng = np.random.default_rng(4)
    samples = W[None] * (1 + 2e-3 * rng.standard_normal((200,) + W.shape))
    res = potential.static_potential(samples)
    assert res["T_plateau"].min() >= 2                 # T = 1 still carries the excited state
    assert np.all(np.diff(res["V"]) > 0)
    assert abs(res["sigma_a2"] - s) < 4 * res["sigma_a2_err"] + 2e-3
    assert 0 < res["sigma_a2_err"] < 0.01
    # the jackknife error of a plain mean is the standard error
    x = rng.standard_normal(400)
    m, e, _ = potential.jackknife(x[:, None], lambda v: v[0])
    assert abs(m - x.mean()) < 1e-12 and abs(e - x.std(ddof=1) / 20) < 1e-12
