"""Pins for the oracle's a0 sampler and single-link heat bath (Section 2, Eqs. 5-9).

Targets fixed by the mathematics, not by the oracle:
  * P(a0) proportional to sqrt(1-a0^2) exp(alpha a0) on [-1,1] (Eq. 8), its CDF
    integrated numerically here;
  * <a0> = I2(alpha)/I1(alpha) (the normaliser is pi I1(alpha)/alpha and its
    alpha-derivative gives the first moment);
  * the vector part of X = U_new W^dagger uniform on the 2-sphere (Eq. 7) and
    independent of a0 (the density exp(beta k x0) dX factorises), in both
    uniform maps; in the 23-bit map cos(theta) lies on the grid of 2^18
    midpoints of [-1, 1].
"""
import numpy as np
import pytest
from scipy import special, stats

import oracle


def target_cdf(alpha):
    x = np.linspace(-1.0, 1.0, 400001)
    f = np.sqrt(np.clip(1.0 - x * x, 0.0, None)) * np.exp(alpha * (x - 1.0))
    F = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(x))])
    F /= F[-1]
    return lambda v: np.interp(v, x, F)


def bessel_mean(alpha):
    return special.ive(2, alpha) / special.ive(1, alpha)


def draw_a0(alpha, sampler, n, seed=5, max_tries=64):
    ch = oracle.chain(1.0, seed=seed, max_tries=max_tries, sampler=sampler)
    out = []
    capped = 0
    for i in range(n):
        k, a0, _ = oracle.sample_a0(ch, alpha, i, i & 3, i >> 2)
        if k == 0:
            capped += 1
        else:
            out.append(a0)
    return np.array(out), capped


@pytest.mark.parametrize("sampler", [oracle.KP, oracle.CREUTZ])
@pytest.mark.parametrize("alpha", [0.5, 2.0, 6.0, 14.4, 50.0])
def test_a0_distribution(alpha, sampler):
    a0, capped = draw_a0(alpha, sampler, 40000)
    assert len(a0) > 30000
    assert np.all(np.abs(a0) <= 1.0)
    ks = stats.kstest(a0, target_cdf(alpha))
    assert ks.pvalue > 1e-3, ks
    m, se = a0.mean(), a0.std() / np.sqrt(len(a0))
    assert abs(m - bessel_mean(alpha)) < 5 * se, (m, bessel_mean(alpha), se)


def test_kp_rejects_a_shifted_target():
    # Power check: the same KS statistic separates alpha from alpha*1.1.
    a0, _ = draw_a0(6.0, oracle.KP, 40000)
    assert stats.kstest(a0, target_cdf(6.6)).pvalue < 1e-6


def _unit(q):
    return q / np.linalg.norm(q)


def _link_samples(u23, nsamp=30000):
    rng = np.random.default_rng(9)
    sigma = 2.3 * _unit(rng.standard_normal(4)) + 0.4 * _unit(rng.standard_normal(4))
    k = np.linalg.norm(sigma)
    beta = 2.1
    ch = oracle.chain(beta, seed=17, u23=u23)
    old = _unit(rng.standard_normal(4))
    a0s, vecs = [], []
    w = sigma / k
    wd = oracle.qdag(w)
    for sweep in range(nsamp):
        n, new, _ = oracle.heatbath_link(ch, 3, 1, sweep, sigma, old)
        assert n > 0
        assert abs(new @ new - 1.0) < 1e-14
        x = oracle.qmul(new, wd)            # X = U_new W^dagger
        a0s.append(new @ sigma / k)         # (1/2) Tr(U_new Sigma^dagger) / k
        assert abs(x[0] - a0s[-1]) < 1e-13
        vecs.append(x[1:] / np.linalg.norm(x[1:]))
    return ch, sigma, old, beta * k, np.array(a0s), np.array(vecs)


def test_single_link_heatbath_distribution(u23=0):
    ch, sigma, old, alpha, a0s, vecs = _link_samples(u23)
    k = np.linalg.norm(sigma)
    wd = oracle.qdag(sigma / k)
    assert stats.kstest(a0s, target_cdf(alpha)).pvalue > 1e-3
    # uniform direction on S^2: mean 0, second moments delta_ij / 3, and
    # each component (= cos of the angle to that axis) uniform on [-1, 1]
    n = len(vecs)
    assert np.all(np.abs(vecs.mean(0)) < 5 / np.sqrt(3 * n))
    M = vecs.T @ vecs / n
    assert np.all(np.abs(M - np.eye(3) / 3) < 5 * np.sqrt(2 / 15 / n) + 1e-3)
    for i in range(3):
        assert stats.kstest(vecs[:, i], stats.uniform(-1, 2).cdf).pvalue > 1e-3
    # independence of a0 and the direction: a 4 x 4 contingency table of a0
    # quartiles against cos(theta) quartiles, and against phi quartiles
    qa = np.searchsorted(np.quantile(a0s, [0.25, 0.5, 0.75]), a0s)
    for comp in (vecs[:, 2], np.arctan2(vecs[:, 1], vecs[:, 0])):
        qc = np.searchsorted(np.quantile(comp, [0.25, 0.5, 0.75]), comp)
        table = np.zeros((4, 4))
        np.add.at(table, (qa, qc), 1)
        assert stats.chi2_contingency(table).pvalue > 1e-3
    # power check: composing with the wrong staple orientation
    # (U = X W^dagger) gives a statistic the same test rejects
    wrong = []
    for sweep in range(3000):
        _, new, _ = oracle.heatbath_link(ch, 3, 1, sweep, sigma, old)
        x = oracle.qmul(new, wd)
        wrong.append(oracle.qmul(x, wd) @ sigma / k)
    assert stats.kstest(np.array(wrong), target_cdf(alpha)).pvalue < 1e-6


def test_single_link_heatbath_distribution_fp32_map():
    test_single_link_heatbath_distribution(u23=1)


def test_fp32_map_direction_grid():
    # 23-bit map: cos(theta) = (2c + 1) 2^-18 - 1 for an integer c < 2^18 (the
    # z component of the unit vector part of X), a grid no 32-bit direction
    # lands on; the 32-bit map's values are off it
    for u23, on_grid in ((1, True), (0, False)):
        *_, vecs = _link_samples(u23, nsamp=400)
        c = ((vecs[:, 2] + 1.0) * 2.0 ** 18 - 1.0) / 2.0
        off = np.abs(c - np.round(c))
        assert np.all(np.round(c) >= 0) and np.all(np.round(c) < 2 ** 18)
        if on_grid:
            assert off.max() < 1e-4, off.max()
        else:
            assert np.median(off) > 0.1


def test_direction_power_check():
    # the contingency test separates a direction that depends on a0: the
    # cos(theta) of X tilted towards a0 fails it
    _, _, _, _, a0s, vecs = _link_samples(1, nsamp=8000)
    z = np.clip(vecs[:, 2] + 0.3 * (a0s - a0s.mean()) / a0s.std(), -1, 1)
    qa = np.searchsorted(np.quantile(a0s, [0.25, 0.5, 0.75]), a0s)
    qc = np.searchsorted(np.quantile(z, [0.25, 0.5, 0.75]), z)
    table = np.zeros((4, 4))
    np.add.at(table, (qa, qc), 1)
    assert stats.chi2_contingency(table).pvalue < 1e-6


def test_haar_branch_and_cap():
    ch = oracle.chain(0.0, seed=3)
    sigma = np.array([0.3, -0.1, 0.2, 0.5])
    old = np.array([1.0, 0.0, 0.0, 0.0])
    n, new, _ = oracle.heatbath_link(ch, 0, 0, 0, sigma, old)
    assert n == -1 and abs(new @ new - 1) < 1e-14
    # beta = 0 draws from the Haar measure: E[a0] = 0, E[a0^2] = 1/4
    qs = np.array([oracle.heatbath_link(ch, s, 0, 0, sigma, old)[1] for s in range(20000)])
    assert abs(qs[:, 0].mean()) < 5 * 0.5 / np.sqrt(len(qs))
    assert abs((qs ** 2).mean(0) - 0.25).max() < 0.02
    # one try at tiny alpha: most links keep their old value, exactly
    ch1 = oracle.chain(1e-3, seed=3, max_tries=1)
    kept = 0
    for s in range(200):
        n, new, _ = oracle.heatbath_link(ch1, s, 2, 5, sigma, old)
        if n == 0:
            kept += 1
            assert np.array_equal(new, old)
    assert kept > 150
