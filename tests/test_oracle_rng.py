"""Pins of the oracle's Philox4x32-10 and Box-Muller normals (CPU only).

The oracle's Philox is written from the published definition (Salmon et al.,
SC'11).  It is pinned bit for bit against the library implementation in
cuRAND's host generator (CURAND_RNG_PSEUDO_PHILOX4_32_10, run on the CPU),
whose raw output block i is the Philox block at counter
(i // 65536, 0, i % 65536, 0) under the key (seed lo32, seed hi32).
"""
import ctypes
import ctypes.util
import math

import numpy as np
import pytest

from oracle import mc

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for name in ("libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            pass
    path = ctypes.util.find_library("curand")
    if path:
        return ctypes.CDLL(path)
    pytest.skip("libcurand not found")


def _curand_host_words(seed, nwords):
    lib = _curand()
    gen = ctypes.c_void_p()
    if lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) != 0:
        pytest.skip("cuRAND host generator unavailable")
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(nwords, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(nwords)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [1234, 0xFEDCBA9876543210, 0xFFFFFFFF00000001])
def test_philox_matches_curand_host_generator(seed):
    n_blocks = 3 * 65536 + 64
    words = _curand_host_words(seed, 4 * n_blocks)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    rng = np.random.default_rng(seed & 0xFFFF)
    idx = sorted(set([0, 1, 2, 65535, 65536, 65537, 2 * 65536 + 5, n_blocks - 1]
                     + list(rng.integers(0, n_blocks, 200))))
    for i in idx:
        ctr = [i // 65536, 0, i % 65536, 0]
        assert mc.philox(ctr, key) == [int(v) for v in words[4 * i:4 * i + 4]], i


def test_stream_layout_key_and_counter():
    seed, inst, sample, call = 0x0123456789ABCDEF, 77, (5 << 32) + 9, 13
    assert mc.philox_words(seed, inst, sample, call) == mc.philox(
        [call, inst, sample & 0xFFFFFFFF, sample >> 32], [seed & 0xFFFFFFFF, seed >> 32])


def _box_muller_ref(words, bits, pair=0):
    """Box-Muller from the raw words, written out in numpy: the 53-bit pair
    from (w0, w1) and (w2, w3); the 24-bit pair `pair` from (w0, w1) or
    (w2, w3)."""
    w = np.asarray(words, dtype=np.uint64)
    if bits == 53:
        u1 = ((w[0] << np.uint64(21)) | (w[1] >> np.uint64(11))).astype(np.float64)
        u2 = ((w[2] << np.uint64(21)) | (w[3] >> np.uint64(11))).astype(np.float64)
        u1, u2 = (u1 + 0.5) * 2.0 ** -53, (u2 + 0.5) * 2.0 ** -53
    else:
        u1 = (np.float32(int(w[2 * pair]) >> 8) + np.float32(0.5)).astype(np.float64) * 2.0 ** -24
        u2 = (np.float32(int(w[2 * pair + 1]) >> 8) + np.float32(0.5)).astype(np.float64) * 2.0 ** -24
    r = math.sqrt(-2.0 * math.log(u1))
    return r * math.cos(2 * math.pi * u2), r * math.sin(2 * math.pi * u2)


def test_normals_follow_box_muller_of_the_stream_53():
    """Double layout: normal j is branch j & 1 of call j >> 1."""
    seed, inst, sample = 99, 3, 12345
    z = mc.normals(seed, inst, sample, 10, 53)
    for t in range(5):
        z0, z1 = _box_muller_ref(mc.philox_words(seed, inst, sample, t), 53)
        assert abs(z[2 * t] - z0) <= 1e-14 * max(1, abs(z0))
        assert abs(z[2 * t + 1] - z1) <= 1e-14 * max(1, abs(z1))


def test_normals_follow_box_muller_of_the_stream_24():
    """Single layout: with j' = j + 1, normal j is branch j' & 1 of pair
    (j' >> 1) & 1 of call j' >> 2 (slot 0 of call 0 unused)."""
    seed, inst, sample = 99, 3, 12345
    n = 23
    z = mc.normals(seed, inst, sample, n, 24)
    for j in range(n):
        jp = j + 1
        pair = mc.philox_words(seed, inst, sample, jp >> 2)
        ref = _box_muller_ref(pair, 24, (jp >> 1) & 1)[jp & 1]
        assert abs(z[j] - ref) <= 1e-14 * max(1, abs(ref)), j
    # from level 3 on (heap index 3, 7, 15, ...) a level starts a call
    for n_lev in range(3, 8):
        j0 = (1 << (n_lev - 1)) - 1
        assert (j0 + 1) % 4 == 0


@pytest.mark.parametrize("bits", [53, 24])
def test_normals_are_standard_normal(bits):
    stats = pytest.importorskip("scipy.stats")
    z = np.concatenate([mc.normals(2024, 0, s, 64, bits) for s in range(800)])
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # the two Box-Muller branches are uncorrelated
    assert abs(np.corrcoef(z[0::2], z[1::2])[0, 1]) < 5 / math.sqrt(z.size / 2)
