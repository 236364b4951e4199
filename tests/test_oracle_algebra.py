"""Pins for the oracle's SU(2) algebra and lattice geometry.

The quaternion product is checked against the explicit 2x2 complex matrix
product of U = q0 1 + i q.sigma (Section 2, Eq. 1), which fixes the sign of
the cross-product term and the order of the factors.
"""
import numpy as np

import oracle
import su2mat


def test_qmul_matches_matrix_product():
    rng = np.random.default_rng(1)
    for _ in range(200):
        a, b = rng.standard_normal(4), rng.standard_normal(4)
        ref = su2mat.to_quat(su2mat.to_mat(a) @ su2mat.to_mat(b))
        np.testing.assert_allclose(oracle.qmul(a, b), ref, atol=1e-14, rtol=0)


def test_qdag_is_conjugate_transpose():
    rng = np.random.default_rng(2)
    for _ in range(50):
        a = rng.standard_normal(4)
        ref = su2mat.to_quat(su2mat.dag(su2mat.to_mat(a)))
        np.testing.assert_allclose(oracle.qdag(a), ref, atol=0, rtol=0)


def test_trace_and_determinant():
    # Tr U = 2 a0 and det U = |a|^2 (Section 2, Eq. 3); det(ab) = det(a) det(b).
    rng = np.random.default_rng(3)
    for _ in range(50):
        a, b = rng.standard_normal(4), rng.standard_normal(4)
        M = su2mat.to_mat(a)
        assert abs(np.trace(M) - 2 * a[0]) < 1e-14
        assert abs(np.linalg.det(M) - a @ a) < 1e-12
        ab = oracle.qmul(a, b)
        assert abs(ab @ ab - (a @ a) * (b @ b)) < 1e-12


def test_shift_and_volume():
    dims = [4, 6, 2, 8]
    assert oracle.volume(dims) == 4 * 6 * 2 * 8
    nd, d = oracle._dims(dims)
    sh = su2mat.shift_table(dims)
    L = oracle.lib()
    for s in range(0, oracle.volume(dims), 7):
        for mu in range(4):
            assert L.oracle_shift(nd, d, s, mu, 1) == sh[s, mu, 0]
            assert L.oracle_shift(nd, d, s, mu, -1) == sh[s, mu, 1]
            # x0 fastest: site index of (x0+1) for x0 < N0-1 is s+1
    assert L.oracle_shift(nd, d, 0, 0, 1) == 1
    assert L.oracle_shift(nd, d, 0, 3, 1) == 4 * 6 * 2
    assert L.oracle_shift(nd, d, 0, 3, -1) == 4 * 6 * 2 * 7
