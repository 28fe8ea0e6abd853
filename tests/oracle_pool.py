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


def _walker_checkpoints(job):
    """One walker's oracle path; the state after every slice listed in
    `checkpoints` as (k, G, ln w, alive, ln det), plus (E_L, N_L) at the end."""
    sysd, fields_w, checkpoints, n = job
    from oracle import afqmc
    from oracle.ueg import UEG
    s = UEG(sysd["N"], sysd["M"], sysd["rs"], sysd["theta"], sysd["dtau"])
    st = afqmc.initial_state(s)
    opts = afqmc.Options()
    keep = set(checkpoints)
    out = []
    for k in range(1, n + 1):
        st, *_ = afqmc.slice_step(s, st, fields_w[k - 1], k, opts)
        if k in keep:
            out.append((k, st.G, st.logw, st.alive, st.logdet))
    E, Nn = afqmc.local_energy(s, st.G)
    return out, (E, Nn)


def _run(fn, jobs):
    # each child gets its share of the cores for BLAS (spawned children read
    # the environment at start-up; oversubscribed BLAS threads spin)
    share = str(max(1, (os.cpu_count() or 1) // len(jobs)))
    saved = {k: os.environ.get(k) for k in _BLAS_VARS}
    os.environ.update({k: share for k in _BLAS_VARS})
    try:
        pool = mp.get_context("spawn").Pool(len(jobs))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return pool, pool.map_async(fn, jobs)


def walkers_mu_fd(sysd, fields, walkers, h=1e-4):
    """Per-walker central differences in mu (fixed draws, frozen force bias)
    for the walkers listed, one process per walker."""
    jobs = [(sysd, np.ascontiguousarray(fields[:, w, :]), h) for w in walkers]
    pool, res = _run(_walker_fd, jobs)
    with pool:
        return res.get()


class Checkpoints:
    """Oracle paths of several walkers, started in the background by the
    constructor; `get` waits for them.  walkers: list of (system dict,
    fields [n][N_alpha]); every path runs n slices and keeps `checkpoints`."""

    def __init__(self, walkers, checkpoints, n):
        jobs = [(sysd, np.ascontiguousarray(f), list(checkpoints), n) for sysd, f in walkers]
        self._pool, self._res = _run(_walker_checkpoints, jobs)

    def get(self, timeout=None):
        try:
            return self._res.get(timeout)
        finally:
            self._pool.close()
            self._pool.join()
