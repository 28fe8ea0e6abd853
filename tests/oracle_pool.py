"""Test infrastructure: runs the CPU oracle on sampled walkers in a process
pool started with 'spawn' (safe after the test process has used the GPU).
Nothing here computes anything itself; it only calls oracle/."""
import multiprocessing as mp
import os

import numpy as np

_BLAS_VARS = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")


def _walker_fd(job):
    sysd, fields_w, h = job
    from oracle import afqmc
    from oracle.ueg import UEG
    s = UEG(sysd["N"], sysd["M"], sysd["rs"], sysd["theta"], sysd["dtau"])
    return afqmc.mu_derivative_walkers_fd(s, fields_w[:, None, :], h=h)[0]


def walkers_mu_fd(sysd, fields, walkers, h=1e-4):
    """Per-walker central differences in mu (fixed draws, frozen force bias)
    for the walkers listed, one process per walker."""
    jobs = [(sysd, np.ascontiguousarray(fields[:, w, :]), h) for w in walkers]
    # each child gets its share of the cores for BLAS (spawned children read
    # the environment at start-up; oversubscribed BLAS threads spin)
    share = str(max(1, (os.cpu_count() or 1) // len(jobs)))
    saved = {k: os.environ.get(k) for k in _BLAS_VARS}
    os.environ.update({k: share for k in _BLAS_VARS})
    try:
        with mp.get_context("spawn").Pool(len(jobs)) as pool:
            return pool.map(_walker_fd, jobs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
