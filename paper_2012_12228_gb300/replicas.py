"""Combination of independent replicas, one process per GPU.

Walkers are independent between population-control events, so every rank
propagates its own walkers with its own fields and the ranks meet only to
combine results (Sec. Computational Details: the estimates come from many
independent simulations).  Each rank's weighted sums from ``ftq_estimators``
carry weights scaled by exp(-s_r), s_r the rank's largest ln|w| over its
alive walkers; the combination rescales every rank to the global largest s
before summing, so the result equals the weighted estimate over the union of
all ranks' walkers.  Works on any torch.distributed backend (NCCL between
GPUs, gloo on CPU); no collective touches the walker data path.
"""
import math


def _dist():
    import torch.distributed as dist
    return dist


def max_over_ranks(x, device=None, group=None):
    """Largest value of the float x over the ranks (x itself without a process group)."""
    dist = _dist()
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def combine_estimates(est, device=None, group=None):
    """Combine the dict returned by ``Propagator.estimators`` over the ranks.

    Returns the same keys (sum_w, sum_wE, sum_wN, log_scale, n_alive, E, N),
    with the sums scaled by exp(-log_scale) for the global log_scale.  A rank
    with no alive walker contributes nothing."""
    dist = _dist()
    if not (dist.is_available() and dist.is_initialized()):
        return dict(est)
    import torch
    alive = int(est["n_alive"]) > 0
    s = torch.tensor([est["log_scale"] if alive else -math.inf], dtype=torch.float64, device=device)
    dist.all_reduce(s, op=dist.ReduceOp.MAX, group=group)
    S = float(s.item())
    f = math.exp(est["log_scale"] - S) if alive and math.isfinite(S) else 0.0
    v = torch.tensor([est["sum_w"].real * f, est["sum_w"].imag * f, est["sum_wE"].real * f, est["sum_wE"].imag * f,
                      est["sum_wN"].real * f, est["sum_wN"].imag * f, float(est["n_alive"])],
                     dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.SUM, group=group)
    v = v.tolist()
    sw, swe, swn = complex(v[0], v[1]), complex(v[2], v[3]), complex(v[4], v[5])
    nan = complex(math.nan, math.nan)
    return dict(sum_w=sw, sum_wE=swe, sum_wN=swn, log_scale=S if math.isfinite(S) else 0.0, n_alive=int(v[6]),
                E=swe / sw if sw != 0 else nan, N=swn / sw if sw != 0 else nan)
