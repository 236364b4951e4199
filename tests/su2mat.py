"""Independent SU(2) algebra for the tests, in explicit 2x2 complex matrices.

U = q0 1 + i (q1 sigma1 + q2 sigma2 + q3 sigma3) (Section 2, Eq. 1).  Nothing
here calls the oracle or the CUDA library: it is the textbook matrix form the
tests pin both against.
"""
import numpy as np

S1 = np.array([[0, 1], [1, 0]], complex)
S2 = np.array([[0, -1j], [1j, 0]], complex)
S3 = np.array([[1, 0], [0, -1]], complex)
ONE = np.eye(2, dtype=complex)


def to_mat(q):
    q = np.asarray(q, float)
    return (q[..., 0, None, None] * ONE + 1j * (q[..., 1, None, None] * S1
            + q[..., 2, None, None] * S2 + q[..., 3, None, None] * S3))


def to_quat(m):
    """Inverse of to_mat for matrices of the form a0 1 + i a.sigma (real a)."""
    q0 = (m[..., 0, 0] + m[..., 1, 1]).real / 2
    q3 = (m[..., 0, 0] - m[..., 1, 1]).imag / 2
    q1 = (m[..., 0, 1] + m[..., 1, 0]).imag / 2
    q2 = (m[..., 0, 1] - m[..., 1, 0]).real / 2
    return np.stack([q0, q1, q2, q3], axis=-1)


def dag(m):
    return np.conj(np.swapaxes(m, -1, -2))


def half_retr(m):
    return (np.trace(m, axis1=-2, axis2=-1).real) / 2


def coords(dims, s):
    x = []
    for n in dims:
        x.append(s % n)
        s = s // n
    return x


def shift_table(dims):
    """shift[s, mu, 0] = s + mu-hat, shift[s, mu, 1] = s - mu-hat (periodic)."""
    V = int(np.prod(dims))
    s = np.arange(V)
    x = coords(dims, s)
    nd = len(dims)
    out = np.empty((V, nd, 2), np.int64)
    for mu in range(nd):
        for k, step in enumerate((1, -1)):
            y = list(x)
            y[mu] = (x[mu] + step) % dims[mu]
            idx = np.zeros(V, np.int64)
            for d in reversed(range(nd)):
                idx = idx * dims[d] + y[d]
            out[:, mu, k] = idx
    return out


def gauge_transform(dims, U, g):
    """U_mu(x) -> g(x) U_mu(x) g(x+mu)^dagger, in matrix form."""
    sh = shift_table(dims)
    G = to_mat(g)
    M = to_mat(U)
    out = np.empty_like(U)
    for mu in range(len(dims)):
        out[:, mu] = to_quat(G @ M[:, mu] @ dag(G[sh[:, mu, 0]]))
    return out
