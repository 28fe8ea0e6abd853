"""Population control between slices (oracle; test infrastructure only, see
oracle/__init__).

The paper controls the walker population with the comb method (Computational
Details; Booth, Thom and Alavi 2009, and the CPMC-Lab description) and names
pair branching for low temperatures without giving either algorithm.  The
comb, from its published definition: with phaseless weights w_i (i < W) and
their running sums C_i, put W teeth at t_k = (k + xi) (S / W) (k < W,
S = C_{W-1}, one uniform draw xi in [0, 1)); walker i receives the teeth in
[C_{i-1}, C_i), i.e. n_i copies, and every copy carries the weight S / W.

Reading (the paper gives no detail): the draw xi is an input; walkers with
n_i >= 1 keep their slot, the extra copies fill the slots of walkers with
n_i = 0 (both taken in ascending order); the weights are rescaled in log form,
ln|w| = ln(S / W) + max_i ln|w_i|, with S over w_i = exp(ln|w_i| - max).
Only the phaseless (real, non-negative) weights are combed.
"""
import math
from dataclasses import replace

import numpy as np

from .afqmc import Options, initial_state, slice_step


def comb_counts(weights, xi):
    """Copies n_i of every walker for the comb with draw xi (sums in index order)."""
    w = np.asarray(weights, dtype=np.float64)
    W = len(w)
    C = np.cumsum(w)                     # running sums, sequential in index order
    step = C[-1] / W
    n = np.zeros(W, dtype=np.int64)
    i = 0
    for k in range(W):
        t = (k + xi) * step
        while i < W - 1 and t >= C[i]:
            i += 1
        n[i] += 1
    return n


def comb_pairs(n):
    """(source, destination) copies: extra copies of walker i (n_i - 1 of them,
    i ascending) go to the walkers with n = 0 (ascending)."""
    empty = [i for i in range(len(n)) if n[i] == 0]
    extra = [i for i in range(len(n)) for _ in range(int(n[i]) - 1)]
    assert len(empty) == len(extra)
    return list(zip(extra, empty))


def scaled_weights(states):
    """(w_i = exp(ln|w_i| - ref), ref) over alive walkers; dead walkers weigh 0."""
    lw = np.array([s.logw.real if s.alive else -np.inf for s in states])
    ref = np.max(lw)
    return np.where(np.isfinite(lw), np.exp(lw - ref), 0.0), ref


def population_control(states, xi):
    """Comb a list of WalkerState; returns (new states, parent of every slot)."""
    W = len(states)
    w, ref = scaled_weights(states)
    if not np.isfinite(ref):
        raise ValueError("no walker alive")
    n = comb_counts(w, xi)
    parent = list(range(W))
    for src, dst in comb_pairs(n):
        parent[dst] = src
    S = np.cumsum(w)[-1]
    lw = math.log(S / W) + ref
    new = [replace(states[parent[i]], logw=complex(lw, 0.0), alive=True) for i in range(W)]
    return new, parent


def run_with_population_control(sys, fields, pc_after, xis, opts: Options = None):
    """All walkers slice by slice; after slice k in `pc_after` the population
    is combed with the next draw of `xis`.  Returns the final states."""
    opts = opts or Options()
    n, W = fields.shape[0], fields.shape[1]
    states = [initial_state(sys) for _ in range(W)]
    draws = iter(xis)
    for k in range(1, n + 1):
        states = [slice_step(sys, st, fields[k - 1, w], k, opts)[0] for w, st in enumerate(states)]
        if k in pc_after:
            states, _ = population_control(states, next(draws))
    return states
