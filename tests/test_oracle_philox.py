"""Pins for the oracle's Philox4x32-10 and uniform conversion (CPU only)."""
import ctypes
import os

import numpy as np
import pytest

from oracle.philox import draw_uniforms, philox4x32_10, words_to_uniform

CURAND_CANDIDATES = ["/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"]


def _curand():
    for p in CURAND_CANDIDATES:
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    return None


@pytest.mark.parametrize("seed", [0, 1234, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    """cuRAND's Philox4_32_10 host generator is an independent implementation of the
    same published algorithm; its block j is Philox at counter (j div 65536, 0,
    j mod 65536, 0) under key (seed lo, seed hi)."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4 * 200000  # spans more than one 65536-block stripe
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    j = np.arange(n // 4, dtype=np.uint64)
    w = philox4x32_10(j // 65536, 0, j % 65536, 0, seed & 0xFFFFFFFF, seed >> 32)
    np.testing.assert_array_equal(np.stack(w, axis=1), out.reshape(-1, 4))


def test_uniform_conversion_exact():
    assert words_to_uniform(0, 0) == 0.0
    top = words_to_uniform(0xFFFFFFFF, 0xFFFFFFFF)
    assert top == 1.0 - 2.0 ** -53 and top < 1.0
    assert words_to_uniform(0x80000000, 0) == 0.5
    # the low 11 bits of the second word are discarded
    assert words_to_uniform(0, 0x7FF) == 0.0 and words_to_uniform(0, 0x800) == 2.0 ** -53


def test_uniforms_are_uniform_and_independent_across_modes():
    t = np.arange(200000, dtype=np.uint64)
    u = draw_uniforms(42, 7, t, 3)
    assert u.min() >= 0.0 and u.max() < 1.0
    for m in range(3):
        h, _ = np.histogram(u[m], bins=64, range=(0, 1))
        e = len(t) / 64
        chi2 = np.sum((h - e) ** 2 / e)
        assert chi2 < 150  # 63 dof; p < 1e-8 beyond this
    # joint 8x8 histogram of modes 0,1 and 1,2 (independence)
    for a, b in [(0, 1), (1, 2), (0, 2)]:
        h, _, _ = np.histogram2d(u[a], u[b], bins=8, range=[[0, 1], [0, 1]])
        e = len(t) / 64
        assert np.sum((h - e) ** 2 / e) < 150
    # different call ids / rows give different streams
    u2 = draw_uniforms(42, 8, t[:1000], 3)
    u3 = draw_uniforms(42, 7, t[:1000], 3, row=1)
    assert not np.any(u2 == u[:, :1000]) and not np.any(u3 == u[:, :1000])


def test_counter_layout_pairs_modes():
    """Draws of 2 or 5+ coordinates: coordinates 2k and 2k+1 share Philox call k (words 0,1
    and 2,3), each a 53-bit uniform."""
    t = np.array([5, 2 ** 33 + 1], dtype=np.uint64)
    for n in (2, 5):
        u = draw_uniforms(99, 3, t, n, row=2)
        for k in range((n + 1) // 2):
            w = philox4x32_10(t & 0xFFFFFFFF, t >> np.uint64(32), k + 256 * 2, 3, 99, 0)
            np.testing.assert_array_equal(u[2 * k], words_to_uniform(w[0], w[1]))
            if 2 * k + 1 < n:
                np.testing.assert_array_equal(u[2 * k + 1], words_to_uniform(w[2], w[3]))


def test_one_call_layout_for_three_and_four_coordinates():
    """Draws of 3 or 4 coordinates: one Philox call (counter word 2 = 256 row), its 128 bits
    (word 0 most significant) cut from the top into chunks of floor(128 / n) bits; checked
    against Python's big-integer arithmetic on the whole 128-bit value."""
    t = np.array([0, 5, 2 ** 33 + 1, 123456789], dtype=np.uint64)
    for n in (3, 4):
        u = draw_uniforms(99, 3, t, n, row=2)
        w = philox4x32_10(t & 0xFFFFFFFF, t >> np.uint64(32), 256 * 2, 3, 99, 0)
        b = 128 // n
        for j in range(len(t)):
            v = (int(w[0][j]) << 96) | (int(w[1][j]) << 64) | (int(w[2][j]) << 32) | int(w[3][j])
            for m in range(n):
                chunk = (v >> (128 - (m + 1) * b)) & ((1 << b) - 1)
                assert u[m][j] == chunk / float(1 << b), (n, j, m)
    # the grid: a chunk of all ones is the largest uniform below 1
    assert float(((1 << 42) - 1) / float(1 << 42)) < 1.0
