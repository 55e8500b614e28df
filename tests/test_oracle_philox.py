"""Pins for the oracle's Philox4x32-10 and its stream layout (CPU only)."""
import ctypes
import ctypes.util

import numpy as np
import pytest
import scipy.stats

from oracle import streams
from oracle.philox import philox4x32_10, seed_to_key


def _load_curand():
    for name in ("libcurand.so.10", "libcurand.so", ctypes.util.find_library("curand")):
        if not name:
            continue
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    return None


_CURAND = _load_curand()
_PHILOX = 161  # CURAND_RNG_PSEUDO_PHILOX4_32_10


def _curand_host_blocks(seed, first_block, nblocks):
    """cuRAND's host-side PHILOX4_32_10 generator (runs on the CPU, no GPU needed)."""
    g = ctypes.c_void_p()
    assert _CURAND.curandCreateGeneratorHost(ctypes.byref(g), _PHILOX) == 0
    try:
        assert _CURAND.curandSetPseudoRandomGeneratorSeed(g, ctypes.c_ulonglong(seed)) == 0
        assert _CURAND.curandSetGeneratorOffset(g, ctypes.c_ulonglong(4 * first_block)) == 0
        out = np.zeros(4 * nblocks, dtype=np.uint32)
        assert _CURAND.curandGenerate(g, out.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.c_size_t(out.size)) == 0
    finally:
        _CURAND.curandDestroyGenerator(g)
    return out.reshape(-1, 4)


@pytest.mark.skipif(_CURAND is None, reason="libcurand not available")
@pytest.mark.parametrize("seed", [0, 7, 2000, 0xFEEDBEEFCAFE1234, 2**64 - 1])
@pytest.mark.parametrize("first_block", [0, 3, 65530, 2**20 + 5, 2**40 + 12345, 2**52 + 65533])
def test_philox_matches_curand_host_generator(seed, first_block):
    # cuRAND's host generator hands block B = first_block + k the counter
    # (B >> 16, B >> 48, B mod 2^16, 0) under key (seed lo, seed hi): counter words 0, 1 and 2
    # and both key words vary across these cases.
    n = 64
    got = _curand_host_blocks(seed, first_block, n)
    B = np.arange(n, dtype=np.uint64) + np.uint64(first_block)
    k0, k1 = seed_to_key(seed)
    ref = np.stack(philox4x32_10(((B >> np.uint64(16)) & np.uint64(0xFFFFFFFF)).astype(np.uint32),
                                 (B >> np.uint64(48)).astype(np.uint32),
                                 (B & np.uint64(0xFFFF)).astype(np.uint32), 0, k0, k1), axis=1)
    np.testing.assert_array_equal(got, ref)


def test_philox_is_a_bijection_sample():
    # distinct counters under one key never collide (Philox is a bijection on the counter)
    c = np.arange(200000, dtype=np.uint32)
    w = philox4x32_10(c, 5, 6, 7, 11, 12)
    packed = (w[0].astype(np.uint64) << np.uint64(32)) | w[1].astype(np.uint64)
    assert np.unique(packed).size == c.size


@pytest.mark.parametrize("dims", [(7, 50, 400), (400, 400, 400), (13, 3, 100, 2)])
def test_ls_samples_uniform_per_mode(dims):
    S = 40000
    idx = streams.ls_sample_indices(2001, 0, 3, 0, S, dims)
    assert np.all(idx[:, 0] == 0)
    for m in range(1, len(dims)):
        col = idx[:, m]
        assert col.min() >= 0 and col.max() < dims[m]
        counts = np.bincount(col, minlength=dims[m])
        chi2 = scipy.stats.chisquare(counts)
        assert chi2.pvalue > 1e-4, (m, chi2)


def test_ls_samples_independent_between_modes():
    dims = (10, 10, 10)
    idx = streams.ls_sample_indices(9, 0, 0, 2, 100000, dims)
    table = np.zeros((10, 10))
    np.add.at(table, (idx[:, 0], idx[:, 1]), 1)
    assert scipy.stats.chi2_contingency(table).pvalue > 1e-4


def test_ls_samples_fresh_per_iteration_mode_and_batch():
    dims = (30, 40, 50, 60, 70, 80)   # order 6: two Philox blocks per sample
    base = streams.ls_sample_indices(1, 0, 0, 1, 500, dims)
    for args in [(1, 0, 1, 1), (1, 0, 0, 2), (1, 1, 0, 1), (2, 0, 0, 1)]:
        other = streams.ls_sample_indices(args[0], args[1], args[2], args[3], 500, dims)
        assert np.mean(base == other) < 0.2
    again = streams.ls_sample_indices(1, 0, 0, 1, 500, dims)
    np.testing.assert_array_equal(base, again)
    # the fifth non-solved mode comes from the second block: still uniform
    counts = np.bincount(streams.ls_sample_indices(3, 0, 0, 0, 80000, dims)[:, 5], minlength=80)
    assert scipy.stats.chisquare(counts).pvalue > 1e-4


def test_fit_samples_uniform_over_entries():
    dims = (5, 6, 7)
    idx = streams.fit_sample_indices(11, 0, 100000, dims)
    flat = idx[:, 0] + 5 * (idx[:, 1] + 6 * idx[:, 2])
    counts = np.bincount(flat, minlength=210)
    assert scipy.stats.chisquare(counts).pvalue > 1e-4


def test_init_values_and_signs():
    A = streams.init_factor(3, 0, 1, 5000, 7)
    assert A.shape == (5000, 7)
    assert A.min() >= 0.0 and A.max() < 1.0
    np.testing.assert_array_equal(A * 2**24, np.floor(A * 2**24))   # exact multiples of 2^-24
    assert abs(A.mean() - 0.5) < 0.01
    d = streams.sign_vector(3, 0, 2, 100000)
    assert set(np.unique(d)) == {-1.0, 1.0}
    assert abs(d.mean()) < 0.02
