"""Pins for the oracle's random numbers (Philox4x32-10 and the uint32 -> (0,1) map).

The oracle's Philox is checked against two cuRAND routines that share no code
with it: the host-side pseudo-random generator of libcurand (PHILOX4_32_10,
whose output block j, for j below 2^16, is Philox(ctr=(0,0,j,0), key=(S_lo, S_hi)) for seed S)
and the block function of cuRAND's device header evaluated on the host.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def _curand():
    for p in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return C.CDLL(p)
        except OSError:
            continue
    return None


def test_philox_vs_curand_host_generator():
    L = _curand()
    if L is None:
        pytest.skip("libcurand not available")
    rng = np.random.default_rng(7)
    seeds = [0, 1, 0xFFFFFFFFFFFFFFFF, 0x0123456789ABCDEF] + [int(x) for x in rng.integers(0, 2**63, 6)]
    for seed in seeds:
        gen = C.c_void_p()
        assert L.curandCreateGeneratorHost(C.byref(gen), 161) == 0  # PHILOX4_32_10
        try:
            assert L.curandSetPseudoRandomGeneratorSeed(gen, C.c_ulonglong(seed)) == 0
            key = [seed & 0xFFFFFFFF, seed >> 32]
            for j in [0, 1, 2, 3] + [int(x) for x in rng.integers(4, 2**16, 4)]:
                assert L.curandSetGeneratorOffset(gen, C.c_ulonglong(4 * j)) == 0
                buf = (C.c_uint32 * 4)()
                assert L.curandGenerate(gen, buf, 4) == 0
                assert oracle.philox([0, 0, j, 0], key) == list(buf), (seed, j)
        finally:
            L.curandDestroyGenerator(gen)


def test_philox_vs_curand_block_function(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "curand_philox_host")
    subprocess.run([nvcc, "-O1", "-o", exe, os.path.join(HERE, "curand_philox_host.cu")],
                   check=True, cwd=str(tmp_path))
    rng = np.random.default_rng(11)
    cases = [[0] * 6, [0xFFFFFFFF] * 6, [1, 0, 0, 0, 0, 0], [0, 1, 0, 0, 0, 0], [0, 0, 0, 1, 0, 0]]
    cases += [[int(x) for x in rng.integers(0, 2**32, 6)] for _ in range(500)]
    text = "\n".join(" ".join(str(v) for v in c) for c in cases) + "\n"
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split("\n")
    for c, line in zip(cases, out):
        ref = [int(v) for v in line.split()]
        assert oracle.philox(c[:4], c[4:]) == ref, c


def test_u01_closed_form():
    # (x + 1/2) 2^-32: endpoints, midpoint, strict bounds.
    assert oracle.u01(0) == 2.0 ** -33
    assert oracle.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -33
    assert oracle.u01(0x80000000) == 0.5 + 2.0 ** -33
    # 23-bit resolution: ((x >> 9) + 1/2) 2^-23
    assert oracle.u01(0, 1) == 2.0 ** -24
    assert oracle.u01(0xFFFFFFFF, 1) == 1.0 - 2.0 ** -24
    assert oracle.u01(0x000001FF, 1) == 2.0 ** -24
    rng = np.random.default_rng(3)
    for x in rng.integers(0, 2**32, 200):
        x = int(x)
        assert oracle.u01(x) == (x + 0.5) / 2.0 ** 32
        assert oracle.u01(x, 1) == ((x >> 9) + 0.5) / 2.0 ** 23


def test_draw_keying():
    # ctr = (s, mu | lattice_id << 2, sweep, draw), key = (seed_lo, seed_hi).
    seed = 0xDEADBEEF12345678
    ch = oracle.chain(2.0, seed=seed, lattice_id=5)
    u = (C.c_double * 4)()
    oracle.lib().oracle_draw(C.byref(ch), 1234, 3, 77, 9, u)
    raw = oracle.philox([1234, 3 | (5 << 2), 77, 9], [seed & 0xFFFFFFFF, seed >> 32])
    assert list(u) == [(x + 0.5) / 2.0 ** 32 for x in raw]
