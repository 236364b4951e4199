"""Pins for the oracle's measurements (Section 2, Eqs. 12-15, 18, 19).

Checked against what the mathematics fixes:
  * the cold start (every link 1) gives plaquette = Polyakov = W(R,T) = 1;
  * U(1)-embedded configurations (links exp(i theta sigma3)) commute, so every
    loop reduces to the cosine of the oriented sum of its angles, computed here
    with numpy from the angles alone: this fixes link orientation, daggers and
    the order of the factors;
  * gauge invariance (observables) and covariance (APE) under random SU(2)
    gauge transformations applied in explicit 2x2 matrix form;
  * centre flip of one time slice (L -> -L, plaquette unchanged);
  * W(1,1) equals the space-time plaquette.
"""
import numpy as np
import pytest

import oracle
import su2mat
from paper_1010_4834_gb300 import inputs


def abelian_plaquettes(dims, th):
    sh = su2mat.shift_table(dims)
    nd = len(dims)
    sp, tm = [], []
    for mu in range(nd):
        for nu in range(mu + 1, nd):
            ang = th[:, mu] + th[sh[:, mu, 0], nu] - th[sh[:, nu, 0], mu] - th[:, nu]
            (tm if nu == nd - 1 else sp).append(np.cos(ang))
    allp = np.concatenate(sp + tm)
    return allp.mean(), (np.concatenate(sp).mean() if sp else 0.0), np.concatenate(tm).mean()


def walk(sh, s, mu, n):
    for _ in range(n):
        s = sh[s, mu, 0]
    return s


def line_angle(sh, th, s, mu, n):
    a = np.zeros(len(s))
    for _ in range(n):
        a += th[s, mu]
        s = sh[s, mu, 0]
    return a


def abelian_wilson(dims, th, rmax, tmax):
    sh = su2mat.shift_table(dims)
    nd = len(dims)
    t = nd - 1
    V = int(np.prod(dims))
    s0 = np.arange(V)
    W = np.zeros((rmax, tmax))
    for R in range(1, rmax + 1):
        for T in range(1, tmax + 1):
            acc = []
            for mu in range(t):
                a = (line_angle(sh, th, s0, mu, R) + line_angle(sh, th, walk(sh, s0, mu, R), t, T)
                     - line_angle(sh, th, walk(sh, s0, t, T), mu, R) - line_angle(sh, th, s0, t, T))
                acc.append(np.cos(a))
            W[R - 1, T - 1] = np.concatenate(acc).mean()
    return W


DIMS = [[4, 4, 4, 4], [4, 6, 2, 8], [6, 4]]


@pytest.mark.parametrize("dims", DIMS)
def test_cold_start_is_one(dims):
    U = oracle.init_cold(dims)
    np.testing.assert_array_equal(oracle.plaquette(dims, U)[[0, 2]], [1.0, 1.0])
    assert oracle.polyakov(dims, U) == 1.0
    np.testing.assert_array_equal(oracle.wilson_loops(dims, U, 2, 2), np.ones((2, 2)))


@pytest.mark.parametrize("dims", DIMS)
def test_abelian_closed_forms(dims):
    th = inputs.abelian_angles(dims, 4)
    U = inputs.abelian_field(th)
    p = oracle.plaquette(dims, U)
    np.testing.assert_allclose(p, abelian_plaquettes(dims, th), atol=1e-14, rtol=0)
    nsig = int(np.prod(dims[:-1]))
    L = np.cos(th[:, -1].reshape(dims[-1], nsig).sum(0)).mean()
    assert abs(oracle.polyakov(dims, U) - L) < 1e-14
    rmax, tmax = min(dims[:-1]), dims[-1]
    np.testing.assert_allclose(oracle.wilson_loops(dims, U, rmax, tmax),
                               abelian_wilson(dims, th, rmax, tmax), atol=1e-13, rtol=0)


@pytest.mark.parametrize("dims", DIMS)
def test_gauge_invariance(dims):
    U = inputs.random_field(dims, 5)
    g = inputs.random_gauge(dims, 6)
    Ug = su2mat.gauge_transform(dims, U, g)
    assert np.abs(Ug - U).max() > 0.1
    np.testing.assert_allclose(oracle.plaquette(dims, Ug), oracle.plaquette(dims, U), atol=1e-13)
    assert abs(oracle.polyakov(dims, Ug) - oracle.polyakov(dims, U)) < 1e-13
    np.testing.assert_allclose(oracle.wilson_loops(dims, Ug, 2, 3), oracle.wilson_loops(dims, U, 2, 3),
                               atol=1e-13)
    # a gauge transform of the cold start: non-trivial links, trivial loops
    Cg = su2mat.gauge_transform(dims, oracle.init_cold(dims), g)
    assert abs(oracle.plaquette(dims, Cg)[0] - 1) < 1e-13
    assert abs(oracle.polyakov(dims, Cg) - 1) < 1e-13


def test_centre_flip_and_w11():
    dims = [4, 4, 4, 6]
    U = inputs.random_field(dims, 8)
    nsig = 64
    F = U.copy()
    F[:nsig, 3] *= -1.0        # U_t(x, t=0) -> -U_t
    assert abs(oracle.polyakov(dims, F) + oracle.polyakov(dims, U)) < 1e-15
    np.testing.assert_allclose(oracle.plaquette(dims, F), oracle.plaquette(dims, U), atol=1e-15)
    np.testing.assert_allclose(oracle.wilson_loops(dims, F, 2, 3), oracle.wilson_loops(dims, U, 2, 3),
                               atol=1e-15)
    assert abs(oracle.wilson_loops(dims, U, 1, 1)[0, 0] - oracle.plaquette(dims, U)[2]) < 1e-15


def test_translation_invariance():
    dims = [4, 6, 4, 4]
    U = inputs.random_field(dims, 9)
    sh = su2mat.shift_table(dims)
    for mu in range(4):
        S = U[sh[:, mu, 0]].copy()
        np.testing.assert_allclose(oracle.plaquette(dims, S), oracle.plaquette(dims, U), atol=1e-14)
        assert abs(oracle.polyakov(dims, S) - oracle.polyakov(dims, U)) < 1e-14
        np.testing.assert_allclose(oracle.wilson_loops(dims, S, 2, 2), oracle.wilson_loops(dims, U, 2, 2),
                                   atol=1e-14)


def abelian_ape(dims, th, alpha):
    sh = su2mat.shift_table(dims)
    nd = len(dims)
    t = nd - 1
    out = inputs.abelian_field(th)
    for mu in range(t):
        z = (1 - alpha) * np.exp(1j * th[:, mu])
        for nu in range(t):
            if nu == mu:
                continue
            xm = sh[:, nu, 1]
            z = z + alpha / 4 * np.exp(1j * (th[:, nu] + th[sh[:, nu, 0], mu] - th[sh[:, mu, 0], nu]))
            z = z + alpha / 4 * np.exp(1j * (-th[xm, nu] + th[xm, mu] + th[sh[xm, mu, 0], nu]))
        z = z / np.abs(z)
        out[:, mu, 0] = z.real
        out[:, mu, 3] = z.imag
    return out


@pytest.mark.parametrize("alpha", [0.0, 0.444, 0.7])
def test_ape_abelian_closed_form(alpha):
    dims = [4, 6, 4, 4]
    th = inputs.abelian_angles(dims, 10)
    U = inputs.abelian_field(th)
    np.testing.assert_allclose(oracle.ape_step(dims, U, alpha), abelian_ape(dims, th, alpha),
                               atol=1e-14, rtol=0)


def test_ape_covariance_identity_and_fixed_point():
    dims = [4, 4, 6, 4]
    U = inputs.random_field(dims, 11)
    g = inputs.random_gauge(dims, 12)
    S = oracle.ape_smear(dims, U, 0.7, 3)
    Sg = oracle.ape_smear(dims, su2mat.gauge_transform(dims, U, g), 0.7, 3)
    np.testing.assert_allclose(Sg, su2mat.gauge_transform(dims, S, g), atol=1e-13)
    np.testing.assert_array_equal(S[:, 3], U[:, 3])                 # time links untouched
    np.testing.assert_allclose(oracle.ape_step(dims, U, 0.0), U, atol=1e-15, rtol=0)  # identity
    C = oracle.init_cold(dims)
    np.testing.assert_allclose(oracle.ape_step(dims, C, 0.7), C, atol=1e-15, rtol=0)  # fixed point
    assert np.abs(np.linalg.norm(S, axis=-1) - 1).max() < 1e-14
