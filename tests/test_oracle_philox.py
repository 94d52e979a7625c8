"""Pins for the oracle's Philox4x32-10 (counter-based RNG, Salmon et al. SC'11).

The paper does not describe its RNG (Sec. 3 only states the Monte Carlo
estimator, Eq. 9); the counter layout (pixel, sample, vertex, group) is a
design reading.  The oracle's generator is pinned to an independent
implementation -- curand's host-side Philox4x32-10 generator, run as a black
box -- and by statistical checks.
"""
import ctypes
import os

import numpy as np
import pytest


def _curand():
    for name in ("libcurand.so", "libcurand.so.10", "/usr/local/cuda/lib64/libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


def test_matches_curand_host_philox(oracle_mod):
    """curand's host Philox4x32-10 generator emits philox(ctr=(0,0,i,0), key=(seed_lo, seed_hi))
    as outputs 4i..4i+3; the oracle must reproduce them bit for bit (all ten rounds,
    both multipliers and the Weyl key schedule are exercised)."""
    cr = _curand()
    if cr is None:
        pytest.skip("libcurand not available")
    for seed in (0x1234567890ABCDEF, 25660, 0xFFFFFFFF00000001):
        gen = ctypes.c_void_p()
        assert cr.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
        assert cr.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4 * 300
        out = np.zeros(n, np.uint32)
        assert cr.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
        cr.curandDestroyGenerator(gen)
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for i in list(range(20)) + [123, 299]:
            got = oracle_mod.philox([0, 0, i, 0], key)
            assert (got == out[4 * i:4 * i + 4]).all(), (seed, i)


def _uniforms(oracle_mod, n, key, word):
    u = np.empty(4 * n)
    for i in range(n):
        ctr = [7, 3, 1, 0]
        ctr[word] = i
        u[4 * i:4 * i + 4] = (oracle_mod.philox(ctr, key) >> 8) * 2.0 ** -24
    return u


@pytest.mark.parametrize("word", [0, 1, 3])
def test_uniformity_chi2(oracle_mod, word):
    """Counting along counter words not covered by curand: 64-bin chi^2 of 8000 uniforms."""
    u = _uniforms(oracle_mod, 2000, [25660, 0], word)
    assert u.min() >= 0.0 and u.max() < 1.0
    h, _ = np.histogram(u, bins=64, range=(0, 1))
    e = len(u) / 64
    chi2 = ((h - e) ** 2 / e).sum()
    # 63 dof: P(chi2 > 110) ~ 2e-4
    assert chi2 < 110, chi2


def test_adjacent_keys_uncorrelated(oracle_mod):
    a = _uniforms(oracle_mod, 2500, [1000, 0], 0)
    b = _uniforms(oracle_mod, 2500, [1001, 0], 0)
    r = np.corrcoef(a, b)[0, 1]
    assert abs(r) < 4.0 / np.sqrt(len(a)), r


def test_counter_words_independent(oracle_mod):
    """Swapping two counter words must change the output (no symmetric use)."""
    key = [5, 9]
    for a, b in [(0, 1), (0, 2), (1, 3), (2, 3)]:
        c1 = [11, 22, 33, 44]
        c2 = list(c1)
        c2[a], c2[b] = c2[b], c2[a]
        assert not (oracle_mod.philox(c1, key) == oracle_mod.philox(c2, key)).all()
