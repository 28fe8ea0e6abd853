"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.

This module holds no arithmetic of the method: it only names the workloads
(system sizes and parameters taken from the paper's computational details)
and draws the standard-normal auxiliary fields x ~ N(0, 1) that both the
oracle and the CUDA path consume bit-for-bit.  Fields are drawn with NumPy's
counter-based Philox bit generator keyed by the seed, in the layout
[slice][walker][alpha] (float64, C order).

`philox_fields` is the host counterpart of the CUDA library's own field
generator (used when no fields are passed): Philox4x32-10 (Salmon, Moraes,
Dror, Shaw, SC'11) and the Box-Muller transform, written here independently
from the published definition so that the two can be compared.
"""
import numpy as np

# name: (N-bar, M, r_s, Theta, dtau, walkers)
WORKLOADS = {
    # N=2 (1 up, 1 down), M=7, r_s=1, Theta=0.5: exact diagonalisation checkable
    "ueg_n2_m7": dict(N=2, M=7, rs=1.0, theta=0.5, dtau=0.05, walkers=64, seed=1235),
    # N=14 (7 up, 7 down), M=57, r_s=1, Theta=0.125
    "ueg_n14_m57": dict(N=14, M=57, rs=1.0, theta=0.125, dtau=0.05, walkers=640, seed=1236),
    # N=14, M=123, r_s=2, Theta=0.25 (chemical-potential gradient workload)
    "ueg_n14_m123": dict(N=14, M=123, rs=2.0, theta=0.25, dtau=0.05, walkers=256, seed=1237),
    # N=66 (33 up, 33 down), M=257, r_s=1, Theta=0.0625, dtau=0.025
    "ueg_n66_m257": dict(N=66, M=257, rs=1.0, theta=0.0625, dtau=0.025, walkers=1024, seed=1239),
}

# Ragged batch: four (N, M) systems, each paired with one (r_s, Theta) so that
# r_s in {0.5, 1, 2} and Theta in {0.0625, 0.125, 0.5} all occur; dtau = 0.05,
# 256 walkers each (paths of 43, 87, 87 and 174 slices).
RAGGED = [
    dict(N=14, M=57, rs=0.5, theta=0.0625, dtau=0.05, walkers=256, seed=1301),
    dict(N=38, M=123, rs=2.0, theta=0.5, dtau=0.05, walkers=256, seed=1302),
    dict(N=54, M=171, rs=1.0, theta=0.125, dtau=0.05, walkers=256, seed=1303),
    dict(N=66, M=257, rs=1.0, theta=0.0625, dtau=0.05, walkers=256, seed=1304),
]


def gaussian_fields(seed, n_slices, walkers, n_alpha, first_slice=0):
    """Standard-normal fields x[k][w][alpha] for slices first_slice..+n_slices.

    Slice k of walker w is drawn from its own Philox stream keyed by
    (seed, k) so that any slice window can be regenerated independently."""
    out = np.empty((n_slices, walkers, n_alpha), dtype=np.float64)
    for i in range(n_slices):
        g = np.random.Generator(np.random.Philox(key=[seed, first_slice + i]))
        out[i] = g.standard_normal((walkers, n_alpha))
    return out


# Philox4x32 round multipliers and key-schedule increments (Salmon et al. 2011)
PHILOX_MUL = (0xD2511F53, 0xCD9E8D57)
PHILOX_WEYL = (0x9E3779B9, 0xBB67AE85)
TWO_PI = 6.283185307179586


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of 32-bit counters (any integer
    dtype, values < 2^32) under the key (k0, k1); returns four uint64 arrays
    holding the 32-bit output words.  Each round multiplies words 0 and 2 by
    the round constants, swaps in the high halves xor'ed with the other words
    and the key; the key advances by the Weyl increments between rounds."""
    mask = np.uint64(0xFFFFFFFF)
    c = [np.asarray(x).astype(np.uint64) for x in (c0, c1, c2, c3)]
    k = [np.uint64(k0), np.uint64(k1)]
    for _ in range(10):
        p0 = np.uint64(PHILOX_MUL[0]) * c[0]
        p1 = np.uint64(PHILOX_MUL[1]) * c[2]
        c = [(p1 >> np.uint64(32)) ^ c[1] ^ k[0], p1 & mask, (p0 >> np.uint64(32)) ^ c[3] ^ k[1], p0 & mask]
        k = [(k[0] + np.uint64(PHILOX_WEYL[0])) & mask, (k[1] + np.uint64(PHILOX_WEYL[1])) & mask]
    return c


def uniform53(lo, hi):
    """(0, 1) double from two 32-bit words: the top 53 bits of (hi << 32 | lo), centred."""
    a = ((hi.astype(np.uint64) << np.uint64(32)) | lo.astype(np.uint64)) >> np.uint64(11)
    return (a.astype(np.float64) + 0.5) * 2.0 ** -53


def philox_fields(seed, n_slices, walkers, n_alpha, first_slice=0, system=0):
    """The library's own fields x[k][w][alpha] for slices first_slice..+n_slices:
    counter (alpha // 2, slice, walker, system), key (seed low, seed high),
    x_{2j} = sqrt(-2 ln u1) cos(2 pi u2), x_{2j+1} = sqrt(-2 ln u1) sin(2 pi u2)."""
    assert n_alpha % 2 == 0
    seed = int(seed)
    j = np.arange(n_alpha // 2, dtype=np.uint64)[None, None, :]
    k = (first_slice + np.arange(n_slices, dtype=np.uint64))[:, None, None]
    w = np.arange(walkers, dtype=np.uint64)[None, :, None]
    shape = (n_slices, walkers, n_alpha // 2)
    c0, c1, c2, c3 = philox4x32_10(np.broadcast_to(j, shape), np.broadcast_to(k, shape), np.broadcast_to(w, shape),
                                   np.full(shape, system, dtype=np.uint64), seed & 0xFFFFFFFF, seed >> 32)
    u1, u2 = uniform53(c0, c1), uniform53(c2, c3)
    r = np.sqrt(-2.0 * np.log(u1))
    t = TWO_PI * u2
    out = np.empty((n_slices, walkers, n_alpha), dtype=np.float64)
    out[:, :, 0::2] = r * np.cos(t)
    out[:, :, 1::2] = r * np.sin(t)
    return out
