"""Pins of the oracle's primitives against things other than itself.

- transforms: brute-force DFT, numpy's FFT, Parseval, round trip
- Philox4x32-10: published known-answer vectors
- the single-precision Box-Muller recipe: accuracy against float64 libm and
  the distribution of the normals it yields
- phi-functions: 50-digit mpmath evaluation and the exact z -> 0 limits
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- transforms
@pytest.mark.parametrize("shape", [(8,), (16,), (8, 16), (8, 8, 8), (2, 4, 8),
                                   (12,), (24,), (48,), (6, 10), (24, 12), (3, 4, 6)])  # not powers of two
def test_fft_matches_bruteforce_dft(oracle_mod, shape):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    for sign in (-1, +1):
        a = oracle_mod.fft_nd(x, sign)
        b = oracle_mod.dft_naive(x, sign)
        assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(b).max())


@pytest.mark.parametrize("shape", [(5,), (6, 10), (3, 4, 5), (16, 8)])
def test_bruteforce_dft_matches_numpy(oracle_mod, shape):
    rng = np.random.default_rng(2)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = np.fft.fftn(x)
    assert np.abs(oracle_mod.dft_naive(x, -1) - ref).max() <= 1e-12 * np.abs(ref).max()
    refi = np.fft.ifftn(x) * x.size
    assert np.abs(oracle_mod.dft_naive(x, +1) - refi).max() <= 1e-12 * np.abs(refi).max()


@pytest.mark.parametrize("shape", [(96,), (48, 48), (24, 96), (192, 12), (80,), (160, 40), (112,), (56, 112)])
def test_fft_of_3x2k_lengths_matches_numpy(oracle_mod, shape):
    """Lattices of p x 2^k points (p = 3, 5, 7): the oracle's split-radix transform
    against numpy's FFT."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = np.fft.fftn(x)
    assert np.abs(oracle_mod.fft_nd(x, -1) - ref).max() <= 1e-12 * np.abs(ref).max()
    refi = np.fft.ifftn(x) * x.size
    assert np.abs(oracle_mod.fft_nd(x, +1) - refi).max() <= 1e-12 * np.abs(refi).max()


def test_fft_parseval_and_roundtrip(oracle_mod):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((32, 64))
    X = oracle_mod.fft_nd(x, -1)
    assert abs(np.sum(np.abs(X) ** 2) / x.size - np.sum(x ** 2)) <= 1e-12 * np.sum(x ** 2)
    back = oracle_mod.fft_nd(X, +1) / x.size
    assert np.abs(back - x).max() <= 1e-14 * np.abs(x).max() * 10
    # delta function -> all ones; single cosine -> two spikes of N/2
    d = np.zeros(16)
    d[0] = 1
    assert np.allclose(oracle_mod.fft_nd(d), np.ones(16))
    c = np.cos(2 * np.pi * 3 * np.arange(16) / 16)
    C = oracle_mod.fft_nd(c)
    assert abs(C[3] - 8) < 1e-12 and abs(C[13] - 8) < 1e-12
    assert np.abs(np.delete(C, [3, 13])).max() < 1e-12


def test_fft_sign_convention(oracle_mod):
    # forward transform uses e^{-2 pi i a n / N}: e^{+2 pi i n/N} lands on a = +1
    n = np.arange(8)
    X = oracle_mod.fft_nd(np.exp(2j * np.pi * n / 8), -1)
    assert abs(X[1] - 8) < 1e-12 and np.abs(np.delete(X, 1)).max() < 1e-12


# -------------------------------------------------------------------- Philox
def _kat():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    return rows


def test_philox_known_answers(oracle_mod):
    rows = _kat()
    assert len(rows) == 3
    for r in rows:
        assert oracle_mod.philox4x32_10(r[0:4], r[4:6]) == r[6:10]


def test_philox_counter_sensitivity(oracle_mod):
    base = oracle_mod.philox4x32_10([1, 2, 3, 4], [5, 6])
    for i in range(4):
        ctr = [1, 2, 3, 4]
        ctr[i] ^= 1
        other = oracle_mod.philox4x32_10(ctr, [5, 6])
        flips = sum(bin(a ^ b).count("1") for a, b in zip(base, other))
        assert 30 < flips < 98  # avalanche: about half of 128 bits change


# --------------------------------------------------------- Box-Muller recipe
def test_recipe_log_accuracy(oracle_mod):
    rng = np.random.default_rng(4)
    ks = np.concatenate([np.arange(1, 2000), rng.integers(1, 2 ** 24 + 1, size=20000),
                         2 ** 24 - np.arange(0, 2000), 2 ** np.arange(0, 25)])
    worst = 0.0
    for k in ks:
        x = np.float32(int(k) * 2.0 ** -24)
        got = oracle_mod.bm_log(float(x))
        ref = math.log(float(x))
        if ref == 0.0:
            assert got == 0.0
            continue
        ulp = np.spacing(np.float32(abs(ref)))
        worst = max(worst, abs(got - ref) / ulp)
    assert worst <= 4.0, worst


def test_recipe_sincos_accuracy(oracle_mod):
    rng = np.random.default_rng(5)
    ks = np.concatenate([np.arange(0, 3000), rng.integers(0, 2 ** 24, size=20000),
                         [2 ** 21, 2 ** 22, 3 * 2 ** 21, 2 ** 23, 2 ** 24 - 1]])
    worst = 0.0
    for k in ks:
        s, c = oracle_mod.bm_sincos_turn(int(k))
        ang = 2 * math.pi * int(k) / 2 ** 24
        worst = max(worst, abs(s - math.sin(ang)), abs(c - math.cos(ang)))
    assert worst <= 2.5e-7, worst


def test_recipe_normals_distribution(oracle_mod):
    from scipy import stats
    z = []
    for i in range(8000):
        z.extend(oracle_mod.normals4(1234, i, 7, 0, 0))
    z = np.array(z, dtype=np.float64)
    n = z.size
    assert abs(z.mean()) < 4 / math.sqrt(n)
    assert abs(z.var() - 1) < 4 * math.sqrt(2 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # pairs are uncorrelated
    zz = z.reshape(-1, 2)
    assert abs(np.mean(zz[:, 0] * zz[:, 1])) < 4 / math.sqrt(zz.shape[0])


def test_recipe_extremes(oracle_mod):
    # u1 = 1 gives radius 0; u1 = 2^-24 gives the largest radius sqrt(48 ln 2)
    z0, z1 = oracle_mod.bm_pair(0xFFFFFFFF, 0)
    assert z0 == 0.0 and z1 == 0.0
    z0, z1 = oracle_mod.bm_pair(0x000000FF, 0)
    assert abs(float(z0) - math.sqrt(48 * math.log(2))) < 2e-6 and z1 == 0.0


# -------------------------------------------------------------- phi-functions
def test_phi_functions_vs_mpmath(oracle_mod):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50

    def ref(z):
        z = mp.mpc(z)
        if z == 0:
            return complex(1), complex(0.5)
        p1 = (mp.exp(z) - 1) / z
        p2 = (mp.exp(z) - 1 - z) / z ** 2
        return complex(p1), complex(p2)

    zs = [1e-12, -1e-9, 1e-5, -0.3, 0.49999, 0.5, -0.50001, 1.0, -2.5, -40.0, -700.0, 3.0,
          0.2 + 0.1j, -0.3 + 0.9j, 0.99j, -1.0 + 1.0j, -5 - 3j, -50 + 200j, 1e-10 + 1e-10j]
    for z in zs:
        p1, p2 = oracle_mod.phi12(z)
        r1, r2 = ref(z)
        assert abs(p1 - r1) <= 2e-15 * max(1, abs(r1)), (z, p1, r1)
        assert abs(p2 - r2) <= 2e-15 * max(1, abs(r2)) * (4 if abs(z) > 1 else 1), (z, p2, r2)


def test_phi_function_limits(oracle_mod):
    p1, p2 = oracle_mod.phi12(0.0)
    assert p1 == 1.0 and p2 == 0.5
    # continuity across the series/direct switch at |z| = 0.5 (real) and 1 (complex)
    # (phi2' is below 1/2 there, so a 2e-12 step moves phi2 by less than 1e-12)
    a = oracle_mod.phi12(0.5 - 1e-12)[1]
    b = oracle_mod.phi12(0.5 + 1e-12)[1]
    assert abs(a - b) < 1e-12 + 1e-15
    a = oracle_mod.phi12(1j * (1 - 1e-12))[1]
    b = oracle_mod.phi12(1j * (1 + 1e-12))[1]
    assert abs(a - b) < 1e-12 + 1e-15
