"""Pins for the oracle's Markov chain (start configurations, substeps, sweeps).

Targets fixed by the mathematics:
  * hot start = Haar links (Section 2, Eq. 4), each rebuilt here from the raw
    Philox words with an independent Box-Muller;
  * the first substep from the cold start sees k = 6 (six identity staples in
    4D), so the new links' a0 follow Eq. 8 with alpha = 6 beta;
  * links of one (direction, parity) class are independent: any visiting
    order gives the same result;
  * 2D: the plaquettes are independent with weight exp(beta/2 Tr P), so
    <(1/2) Tr P> = I2(beta)/I1(beta) exactly (up to torus corrections that
    vanish like u^V);
  * 4D strong coupling: <P> = u + 4 u^5 + ..., u = I2(beta)/I1(beta);
  * beta = 0: Haar links, <P> = 0;  large beta: <P> -> 1 - 3/(4 beta);
  * over-relaxation (Eq. 10) keeps the action and is an involution.
"""
import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_1010_4834_gb300 import inputs


def u_ratio(beta):
    return special.ive(2, beta) / special.ive(1, beta)


def binned_mean(x, nbins=20):
    x = np.asarray(x)
    b = x[: len(x) // nbins * nbins].reshape(nbins, -1).mean(1)
    return b.mean(), b.std(ddof=1) / np.sqrt(nbins)


def test_hot_start_from_raw_philox():
    dims = [4, 4, 2, 6]
    seed = 0xABCDEF0123
    ch = oracle.chain(1.0, seed=seed, lattice_id=2)
    U = oracle.init_hot(dims, ch)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for s in range(0, oracle.volume(dims), 5):
        for mu in range(4):
            r = oracle.philox([s, mu | (2 << 2), 0xFFFFFFFF, 0], key)
            u = [(x + 0.5) / 2 ** 32 for x in r]
            z = np.array([np.sqrt(-2 * np.log(u[0])) * np.cos(2 * np.pi * u[1]),
                          np.sqrt(-2 * np.log(u[0])) * np.sin(2 * np.pi * u[1]),
                          np.sqrt(-2 * np.log(u[2])) * np.cos(2 * np.pi * u[3]),
                          np.sqrt(-2 * np.log(u[2])) * np.sin(2 * np.pi * u[3])])
            np.testing.assert_allclose(U[s, mu], z / np.linalg.norm(z), atol=1e-15, rtol=0)


def test_hot_start_is_haar():
    dims = [8, 8, 8, 8]
    U = oracle.init_hot(dims, oracle.chain(1.0, seed=1)).reshape(-1, 4)
    n = len(U)
    assert np.abs(np.einsum("ij,ij->i", U, U) - 1).max() < 1e-14
    assert np.abs(U.mean(0)).max() < 5 * 0.5 / np.sqrt(n)
    M = U.T @ U / n
    assert np.abs(M - np.eye(4) / 4).max() < 5 * np.sqrt(1 / 8 - 1 / 16) / np.sqrt(n)
    assert abs((U[:, 0] ** 4).mean() - 1 / 8) < 0.005       # E[x^4] = 3/(d(d+2)), d = 4
    assert abs(oracle.plaquette(dims, U.reshape(-1, 4, 4))[0]) < 0.02


def test_first_substep_from_cold_start():
    dims = [8, 8, 8, 8]
    beta = 0.4
    U = oracle.init_cold(dims)
    nd, d = oracle._dims(dims)
    assert np.array_equal(oracle.staple(dims, U, 17, 0), [6.0, 0, 0, 0])
    st = oracle.substep(dims, U, oracle.chain(beta, seed=1), 0, 0, 0)
    assert st.updates == oracle.volume(dims) // 2
    x = np.arange(oracle.volume(dims))
    par = (x % 8 + x // 8 % 8 + x // 64 % 8 + x // 512) % 2
    a0 = U[par == 0, 0, 0]
    x0 = np.linspace(-1, 1, 200001)
    f = np.sqrt(np.clip(1 - x0 ** 2, 0, None)) * np.exp(6 * beta * (x0 - 1))
    F = np.concatenate([[0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(x0))])
    assert stats.kstest(a0, lambda v: np.interp(v, x0, F / F[-1])).pvalue > 1e-3
    # the untouched classes are still exactly 1
    assert np.all(U[par == 1, 0, 0] == 1.0) and np.all(U[:, 1:, 0] == 1.0)


def test_substep_order_independence():
    dims = [4, 6, 4, 4]
    ch = oracle.chain(2.3, seed=4, max_tries=3)
    U0 = inputs.random_field(dims, 13)
    for mu in range(4):
        for p in range(2):
            A = U0.copy()
            oracle.substep(dims, A, ch, 9, mu, p)
            B = U0.copy()
            V = oracle.volume(dims)
            for s in reversed(range(V)):
                x = np.array([s % 4, s // 4 % 6, s // 24 % 4, s // 96])
                if x.sum() % 2 != p:
                    continue
                sig = oracle.staple(dims, B, s, mu)
                n, new, _ = oracle.heatbath_link(ch, s, mu, 9, sig, B[s, mu].copy())
                B[s, mu] = new
            np.testing.assert_array_equal(A, B)
            assert np.abs(A - U0).max() > 0.1


def run_chain(dims, beta, ntherm, nmeas, seed=1, sampler=oracle.KP, start="hot"):
    ch = oracle.chain(beta, seed=seed, sampler=sampler)
    U = oracle.init_hot(dims, ch) if start == "hot" else oracle.init_cold(dims)
    meas = []
    for sw in range(ntherm + nmeas):
        oracle.sweep(dims, U, ch, sw)
        if sw >= ntherm:
            meas.append(oracle.plaquette(dims, U)[0])
    return np.array(meas)


@pytest.mark.parametrize("beta", [0.7, 2.0, 5.0])
def test_2d_exact_plaquette(beta):
    p = run_chain([32, 32], beta, 40, 2000, sampler=oracle.CREUTZ if beta < 1 else oracle.KP)
    m, e = binned_mean(p)
    assert abs(m - u_ratio(beta)) < 4 * e + 1e-4, (m, e, u_ratio(beta))


def test_2d_exact_plaquette_has_power():
    # the same statistics separate beta from 1.02 beta
    p = run_chain([32, 32], 2.0, 40, 2000)
    m, e = binned_mean(p)
    assert abs(m - u_ratio(2.04)) > 4 * e


def test_4d_strong_coupling():
    beta = 0.5
    p = run_chain([4, 4, 4, 4], beta, 50, 3000, sampler=oracle.CREUTZ)
    m, e = binned_mean(p)
    u = u_ratio(beta)
    assert abs(m - (u + 4 * u ** 5)) < 4 * e, (m, e, u)


def test_4d_beta_zero_is_haar():
    ch = oracle.chain(0.0, seed=2)
    dims = [4, 4, 4, 4]
    U = oracle.init_cold(dims)
    st = oracle.sweep(dims, U, ch, 0)
    assert st.haar == st.updates == 4 * 256
    vals = []
    for sw in range(1, 40):
        oracle.sweep(dims, U, ch, sw)
        vals.append(oracle.plaquette(dims, U)[0])
    m, e = binned_mean(vals, 13)
    assert abs(m) < 4 * e + 1e-3


def test_4d_weak_coupling():
    beta = 10.0
    p = run_chain([4, 4, 4, 4], beta, 30, 100, start="cold")
    assert abs(p.mean() - (1 - 3 / (4 * beta))) < 0.01


def test_overrelaxation_keeps_action_and_is_involution():
    dims = [4, 4, 4, 4]
    U = inputs.random_field(dims, 14)
    ch = oracle.chain(2.4, seed=1)
    for sw in range(3):
        oracle.sweep(dims, U, ch, sw)
    V = oracle.volume(dims)
    for mu in range(4):
        for p in range(2):
            before = oracle.plaquette(dims, U)[0]
            A = U.copy()
            oracle.overrelax_substep(dims, A, mu, p)
            assert np.abs(A - U).max() > 1e-3
            assert abs(oracle.plaquette(dims, A)[0] - before) < 1e-13
            B = A.copy()
            oracle.overrelax_substep(dims, B, mu, p)
            np.testing.assert_allclose(B, U, atol=1e-13)
            U = A
    assert V == 256


def test_all_cores_build_runs_the_same_chain():
    # the OpenMP build shares the sites of each (direction, parity) class
    # among threads; since those links do not enter each other's staples the
    # result and the counts are those of the serial build, bit for bit
    dims = [6, 4, 8, 4]
    ch = oracle.chain(2.3, seed=5, max_tries=3)
    U = oracle.init_hot(dims, ch)
    A = U.copy()
    sa = [oracle.sweep(dims, A, ch, sw) for sw in range(3)]
    B = U.copy()
    with oracle.parallel():
        assert oracle.threads() >= 1
        sb = [oracle.sweep(dims, B, ch, sw) for sw in range(3)]
    assert oracle.threads() == 1
    np.testing.assert_array_equal(A, B)
    for x, y in zip(sa, sb):
        assert (x.updates, x.trials, x.capped, x.haar) == (y.updates, y.trials, y.capped, y.haar)
    assert sum(x.capped for x in sa) > 0
