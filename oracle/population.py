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

Pair branching (the paper's choice for Theta <= 0.25, citing QWalk), read as:
with weights normalised to their mean, u_i = w_i / (S / W), the heavy walkers
(u > 2, by decreasing u, ties to the lower index) are paired in turn with the
light ones (u < 1/2, by increasing u, ties to the lower index); pair k keeps
the heavy walker a with probability u_a / (u_a + u_b) (draw xi_k < that
ratio), else the light walker b; the kept walker is copied into the other
slot and both carry (w_a + w_b) / 2.  Unpaired walkers keep their weights.
The total weight is conserved exactly and each state's expected weight is
unchanged.
"""
import math
from dataclasses import replace

import numpy as np

from .afqmc import Options, initial_state, slice_step


def comb_counts(weights, xi):
    """Copies n_i of every walker for the comb with draw xi (sums in index order).
    A tooth that rounding places at or beyond S goes to the last walker whose
    weight is above 0 (never to a dead walker)."""
    w = np.asarray(weights, dtype=np.float64)
    W = len(w)
    C = np.cumsum(w)                     # running sums, sequential in index order
    step = C[-1] / W
    last = int(np.nonzero(w > 0)[0][-1])
    n = np.zeros(W, dtype=np.int64)
    i = 0
    for k in range(W):
        t = (k + xi) * step
        while i < last and t >= C[i]:
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
    lw = np.array([s.logw.real if s.alive and math.isfinite(s.logw.real) else -np.inf for s in states])
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


def pair_branch_pairs(weights, draws, high=2.0, low=0.5):
    """(source, destination, new weight) of every pair for pair branching."""
    w = np.asarray(weights, dtype=np.float64)
    W = len(w)
    mean = np.cumsum(w)[-1] / W
    u = w / mean
    heavy = sorted((i for i in range(W) if u[i] > high), key=lambda i: (-u[i], i))
    light = sorted((i for i in range(W) if u[i] < low), key=lambda i: (u[i], i))
    out = []
    for k, (a, b) in enumerate(zip(heavy, light)):
        keep_a = draws[k] < u[a] / (u[a] + u[b])
        src, dst = (a, b) if keep_a else (b, a)
        out.append((src, dst, 0.5 * (w[a] + w[b])))
    return out


def pair_branch(states, draws):
    """Pair branching of a list of WalkerState with the uniform draws (one per
    pair, at least W // 2 of them); returns (new states, parent of every slot)."""
    W = len(states)
    w, ref = scaled_weights(states)
    if not np.isfinite(ref):
        raise ValueError("no walker alive")
    parent = list(range(W))
    new = list(states)
    for src, dst, nw in pair_branch_pairs(w, draws):
        lw = complex(math.log(nw) + ref, 0.0)
        new[src] = replace(states[src], logw=lw, alive=True)
        new[dst] = replace(states[src], logw=lw, alive=True)
        parent[dst] = src
    return new, parent


def run_with_population_control(sys, fields, pc_after, xis, opts: Options = None, method="comb"):
    """All walkers slice by slice; after slice k in `pc_after` the population
    is combed (method "comb": the next draw of `xis`) or pair-branched
    ("pair": the next array of draws).  Returns the final states."""
    opts = opts or Options()
    n, W = fields.shape[0], fields.shape[1]
    states = [initial_state(sys) for _ in range(W)]
    draws = iter(xis)
    for k in range(1, n + 1):
        states = [slice_step(sys, st, fields[k - 1, w], k, opts)[0] for w, st in enumerate(states)]
        if k in pc_after:
            step = population_control if method == "comb" else pair_branch
            states, _ = step(states, next(draws))
    return states
