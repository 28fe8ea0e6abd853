"""Report (test infrastructure, oracle only): the gap between the two mu
derivatives of reading Q on the N=14, M=123, r_s=2, Theta=0.25 workload.

The library accumulates d<N>/dmu and d<E>/dmu at fixed draws with every
slice's force bias held at its value on the path (frozen_bias=True).  The
oracle's mu_derivative_fd can also let the force bias follow mu
(frozen_bias=False).  This script evaluates both by central differences
(h = 1e-4) on the same walkers and prints them and their difference.

    python -m oracle.report_mu_gap [walkers] [processes]
"""
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _one(job):
    sysd, f, frozen = job
    from oracle import afqmc
    from oracle.ueg import UEG
    s = UEG(sysd["N"], sysd["M"], sysd["rs"], sysd["theta"], sysd["dtau"])
    r = afqmc.mu_derivative_fd(s, f[:, None, :], afqmc.Options(), h=1e-4, frozen_bias=frozen)
    return r["dN"], r["dE"], r["N"], r["E"], r["excluded"]


def main():
    from synthetic_inputs import WORKLOADS, gaussian_fields
    from oracle.ueg import UEG
    c = WORKLOADS["ueg_n14_m123"]
    W = int(sys.argv[1]) if len(sys.argv) > 1 else 8
    procs = int(sys.argv[2]) if len(sys.argv) > 2 else min(W, os.cpu_count() or 1)
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    f = gaussian_fields(c["seed"], s.n_slices, W, s.N_alpha)
    jobs = [(c, np.ascontiguousarray(f[:, w, :]), fr) for fr in (True, False) for w in range(W)]
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_one, jobs)
    frozen, follow = np.array(res[:W]), np.array(res[W:])
    print(f"N=14 M=123 r_s=2 Theta=0.25, {s.n_slices} slices, {W} walkers (one walker per estimate), h = 1e-4")
    for w in range(W):
        print(f"walker {w}: dN/dmu frozen {frozen[w, 0]:.6f} following {follow[w, 0]:.6f}; "
              f"dE/dmu frozen {frozen[w, 1]:.6f} following {follow[w, 1]:.6f}")
    dn = np.abs(frozen[:, 0] - follow[:, 0]) / np.abs(follow[:, 0])
    de = np.abs(frozen[:, 1] - follow[:, 1]) / np.maximum(1e-12, np.abs(follow[:, 1]))
    print(f"relative gap: dN/dmu median {np.median(dn):.3e} max {dn.max():.3e}; "
          f"dE/dmu median {np.median(de):.3e} max {de.max():.3e}")


if __name__ == "__main__":
    main()
