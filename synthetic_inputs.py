"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.

This module holds no arithmetic of the method: it only names the workloads
(system sizes and parameters taken from the paper's computational details)
and draws the standard-normal auxiliary fields x ~ N(0, 1) that both the
oracle and the CUDA path consume bit-for-bit.  Fields are drawn with NumPy's
counter-based Philox bit generator keyed by the seed, in the layout
[slice][walker][alpha] (float64, C order).
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
