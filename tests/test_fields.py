"""The host Philox4x32-10 / Box-Muller field generator (the counterpart of the
library's on-device generator), checked against what the definition fixes:
uniform output words, full diffusion of counter and key bits after ten
rounds, standard-normal fields, and window / seed / system independence."""
import numpy as np
import pytest

from synthetic_inputs import philox4x32_10, philox_fields, uniform53

stats = pytest.importorskip("scipy.stats")


def _words(n, key=(12345, 678)):
    i = np.arange(n, dtype=np.uint64)
    return philox4x32_10(i & np.uint64(0xFFFF), i >> np.uint64(16), np.full(n, 3, np.uint64), np.zeros(n, np.uint64),
                         *key)


def test_output_words_are_uniform():
    w = np.concatenate(_words(1 << 18))
    assert w.max() < (1 << 32)
    counts = np.bincount((w >> np.uint64(24)).astype(np.int64), minlength=256)
    chi2, p = stats.chisquare(counts)
    assert p > 1e-4
    bits = np.array([((w >> np.uint64(b)) & np.uint64(1)).mean() for b in range(32)])
    sigma = 0.5 / np.sqrt(w.size)
    assert np.all(np.abs(bits - 0.5) < 6 * sigma)


def test_counter_and_key_bits_diffuse():
    """Flipping one input bit changes half of the 128 output bits on average
    (a round missing a multiply or an xor leaves whole words unchanged)."""
    rng = np.random.default_rng(5)
    n = 2000
    c = [rng.integers(0, 1 << 32, n, dtype=np.uint64) for _ in range(4)]
    k0, k1 = 0x1234ABCD, 0x0F0F0F0F
    base = philox4x32_10(*c, k0, k1)

    def flips(out):
        """Number of output bits (of 128) that differ from the base output, per counter."""
        x = (np.stack(out) ^ np.stack(base)).astype(np.uint32)          # [4][n]
        return np.unpackbits(x.T.copy().view(np.uint8), axis=1).sum(axis=1)

    for word in range(4):
        for bit in (0, 13, 31):
            cc = [x.copy() for x in c]
            cc[word] ^= np.uint64(1 << bit)
            m = flips(philox4x32_10(*cc, k0, k1)).mean()
            assert 62 < m < 66, (word, bit, m)
    for kk in ((k0 ^ 1, k1), (k0, k1 ^ (1 << 31))):
        m = flips(philox4x32_10(*c, *kk)).mean()
        assert 62 < m < 66


def test_uniform53_open_interval():
    lo = np.array([0, 0xFFFFFFFF], dtype=np.uint64)
    hi = np.array([0, 0xFFFFFFFF], dtype=np.uint64)
    u = uniform53(lo, hi)
    assert u[0] == 0.5 * 2.0 ** -53 and u[1] == 1.0 - 0.5 * 2.0 ** -53


def test_fields_are_standard_normal():
    x = philox_fields(20261203, 40, 64, 400)
    flat = x.ravel()
    n = flat.size
    assert abs(flat.mean()) < 5 / np.sqrt(n)
    assert abs(flat.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs(stats.skew(flat)) < 5 * np.sqrt(6 / n)
    assert abs(stats.kurtosis(flat)) < 5 * np.sqrt(24 / n)
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    # the two members of a Box-Muller pair are uncorrelated
    r = np.corrcoef(x[:, :, 0::2].ravel(), x[:, :, 1::2].ravel())[0, 1]
    assert abs(r) < 5 / np.sqrt(n / 2)


def test_windows_seeds_and_systems():
    full = philox_fields(99, 8, 5, 12)
    assert np.array_equal(philox_fields(99, 3, 5, 12, first_slice=5), full[5:8])
    assert not np.allclose(philox_fields(100, 8, 5, 12), full)
    assert not np.allclose(philox_fields(99, 8, 5, 12, system=1), full)
    assert not np.allclose(philox_fields(99 + (1 << 32), 8, 5, 12), full)
