"""Seeded synthetic inputs shared by the tests and the benchmark.

This module holds none of the method's arithmetic: it only draws random
numbers with numpy's seeded generators and arranges them in the canonical
host layout U[s, mu, c] (s = x0 + N0*(x1 + N1*(x2 + N2*x3)), quaternion
components c = 0..3).  The random numbers the heat bath itself draws come from
Philox inside each implementation, not from here.
"""
import numpy as np


def volume(dims):
    return int(np.prod(dims))


def random_unit_quaternions(n, rng):
    """n quaternions uniform on S^3 (normalised isotropic Gaussians)."""
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def random_field(dims, seed):
    """A configuration with every link drawn independently and uniformly on SU(2)."""
    rng = np.random.default_rng(seed)
    nd = len(dims)
    return random_unit_quaternions(volume(dims) * nd, rng).reshape(volume(dims), nd, 4)


def abelian_angles(dims, seed):
    """Angles theta[s, mu] uniform in [-pi, pi)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-np.pi, np.pi, size=(volume(dims), len(dims)))


def abelian_field(theta):
    """Links (cos theta, 0, 0, sin theta): the U(1) subgroup exp(i theta sigma_3)."""
    U = np.zeros(theta.shape + (4,))
    U[..., 0] = np.cos(theta)
    U[..., 3] = np.sin(theta)
    return U


def random_gauge(dims, seed):
    """One uniformly random SU(2) element per site, shape (V, 4)."""
    return random_unit_quaternions(volume(dims), np.random.default_rng(seed))


def batch_betas(n, seed, lo=2.0, hi=2.8):
    """n couplings uniform in [lo, hi) for a batch of independent lattices."""
    return np.random.default_rng(seed).uniform(lo, hi, size=n)
