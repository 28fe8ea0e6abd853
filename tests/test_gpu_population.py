"""Comb population control on the GPU (ftq_population_control) against the
oracle's comb (oracle.population): the same parent of every slot for the
same weights and draw, the same rescaled weights, and whole paths with
combing steps equal to the oracle's (complex128, 1e-10) and to the
complex128 GPU path (mixed precision)."""
import math

import numpy as np
import pytest

from oracle.population import comb_counts, comb_pairs, run_with_population_control
from oracle.ueg import UEG
from synthetic_inputs import WORKLOADS, gaussian_fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ftq():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2012_12228_gb300 as m
    return m


def make(ftq, wl, W, **kw):
    c = WORKLOADS[wl]
    return ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, **kw)


def oracle_parents(lw, alive, xi):
    """Parent map and new ln|w| of the oracle's comb for given weights, and the
    smallest distance of a tooth to a running sum (relative to S / W)."""
    ref = np.max(np.where(alive, lw, -np.inf))
    w = np.where(alive, np.exp(lw - ref), 0.0)
    n = comb_counts(w, xi)
    parent = list(range(len(w)))
    for s, d in comb_pairs(n):
        parent[d] = s
    C = np.cumsum(w)
    S, W = C[-1], len(w)
    teeth = (np.arange(W) + xi) * (S / W)
    margin = np.min(np.abs(teeth[:, None] - C[None, :])) / (S / W)
    return np.array(parent), math.log(S / W) + ref, margin


@pytest.mark.parametrize("xi", [0.0, 0.31, 0.97])
def test_parents_and_weights_match_oracle(ftq, xi):
    p = make(ftq, "ueg_n2_m7", 64)
    s = UEG(2, 7, 1.0, 0.5, 0.05)
    p.propagate(torch.from_numpy(gaussian_fields(21, 12, 64, p.n_alpha)).cuda())
    ws = p.weights().cpu().numpy()
    lw, alive = ws[:, 0], ws[:, 2] > 0.5
    ref_parent, ref_lw, margin = oracle_parents(lw, alive, xi)
    assert margin > 1e-9          # no tooth within rounding of a running sum
    parent = p.population_control(xi).cpu().numpy()
    assert np.array_equal(parent, ref_parent)
    ws2 = p.weights().cpu().numpy()
    assert np.all(ws2[:, 2] > 0.5)
    assert np.max(np.abs(ws2[:, 0] - ref_lw)) < 1e-12 * max(1.0, abs(ref_lw))
    moved = parent != np.arange(64)
    assert np.all(ws2[moved, 3] == ws[parent[moved], 3])     # ln det record copied
    assert p.status() == 0
    p.close()


def test_path_with_combing_matches_oracle_fp64(ftq):
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 32
    f = gaussian_fields(c["seed"], s.n_slices, W, s.N_alpha)
    ref = run_with_population_control(s, f, pc_after={10, 15}, xis=(0.3, 0.77))
    p = make(ftq, "ueg_n2_m7", W)
    fd = torch.from_numpy(f).cuda()
    p.propagate(fd[:10].contiguous())
    p.population_control(0.3)
    p.propagate(fd[10:15].contiguous())
    p.population_control(0.77)
    p.propagate(fd[15:].contiguous())
    G = p.green().cpu().numpy()
    ws = p.weights().cpu().numpy()
    for w in range(W):
        assert np.abs(G[w] - ref[w].G).max() < 1e-10 * np.abs(ref[w].G).max()
        assert bool(ws[w, 2] > 0.5) == ref[w].alive
        if ref[w].alive:
            assert abs(ws[w, 0] - ref[w].logw.real) < 1e-10 * max(1.0, abs(ref[w].logw.real))
    with pytest.raises(ftq.FTQError):
        p.mu_grad()                                           # refused after a comb
    p.reset()
    p.propagate(fd)
    p.mu_grad()                                               # allowed again after reset
    p.close()


def test_mixed_path_with_combing_matches_fp64(ftq):
    c = WORKLOADS["ueg_n14_m57"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 16
    fd = torch.from_numpy(gaussian_fields(c["seed"], 15, W, s.N_alpha)).cuda()
    out = {}
    for prec in (ftq.FTQ_FP64, ftq.FTQ_MIXED):
        p = make(ftq, "ueg_n14_m57", W, precision=prec)
        p.propagate(fd[:5].contiguous())
        par1 = p.population_control(0.45).cpu().numpy()
        p.propagate(fd[5:15].contiguous())
        out[prec] = (par1, p.green().cpu().numpy(), p.weights().cpu().numpy())
        assert p.status() == 0
        p.close()
    a, b = out[ftq.FTQ_FP64], out[ftq.FTQ_MIXED]
    assert np.array_equal(a[0], b[0])
    assert np.abs(a[1] - b[1]).max() < 1e-5 * np.abs(a[1]).max()
    # ln|w| telescopes to 2 ln det(I + A_k) (after the comb, from the comb's
    # common weight): its error is twice that of the FP32 ln det, held to
    # 1e-5 relative
    assert np.max(np.abs(a[2][:, 0] - b[2][:, 0])) < 2e-5 * max(1.0, np.max(np.abs(a[2][:, 3])))


def test_rejected_arguments(ftq):
    p = make(ftq, "ueg_n2_m7", 8)
    with pytest.raises(ftq.FTQError):
        p.population_control(1.0)
    with pytest.raises(ftq.FTQError):
        p.population_control(-0.1)
    p.close()
    q = make(ftq, "ueg_n2_m7", 8, constraint=ftq.FTQ_FREE)
    with pytest.raises(ftq.FTQError):
        q.population_control(0.5)
    q.close()


# ------------------------------------------------------------------ pair branching
def oracle_pair_parents(lw, alive, draws):
    from oracle.population import pair_branch_pairs
    ref = np.max(np.where(alive, lw, -np.inf))
    w = np.where(alive, np.exp(lw - ref), 0.0)
    W = len(w)
    parent = np.arange(W)
    new_lw = np.where(alive, lw, np.nan)
    pairs = pair_branch_pairs(w, draws)
    for src, dst, nw in pairs:
        parent[dst] = src
        new_lw[src] = new_lw[dst] = math.log(nw) + ref
    u = w / (np.cumsum(w)[-1] / W)
    margin = min(np.min(np.abs(u - 2.0)), np.min(np.abs(u[u > 0] - 0.5)))
    for k, (src, dst, _) in enumerate(pairs):
        a, b = (src, dst) if u[src] > 2 else (dst, src)
        margin = min(margin, abs(draws[k] - u[a] / (u[a] + u[b])))
    return parent, new_lw, margin, len(pairs)


def test_pair_branch_matches_oracle(ftq):
    p = make(ftq, "ueg_n14_m57", 64)
    p.propagate(torch.from_numpy(gaussian_fields(23, 30, 64, p.n_alpha)).cuda())
    ws = p.weights().cpu().numpy()
    lw, alive = ws[:, 0], ws[:, 2] > 0.5
    draws = np.random.default_rng(2).random(32)
    ref_parent, ref_lw, margin, npairs = oracle_pair_parents(lw, alive, draws)
    assert margin > 1e-9 and npairs > 0
    parent = p.pair_branch(draws).cpu().numpy()
    assert np.array_equal(parent, ref_parent)
    ws2 = p.weights().cpu().numpy()
    touched = np.isfinite(ref_lw)
    assert np.max(np.abs(ws2[touched, 0] - ref_lw[touched])) < 1e-12 * max(1.0, np.max(np.abs(ref_lw[touched])))
    assert p.status() == 0
    p.close()


def test_path_with_pair_branching_matches_oracle_fp64(ftq):
    c = WORKLOADS["ueg_n14_m57"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W, n = 24, 30
    f = gaussian_fields(c["seed"], n, W, s.N_alpha)
    rng = np.random.default_rng(6)
    d1, d2 = rng.random(W // 2), rng.random(W // 2)
    ref = run_with_population_control(s, f, pc_after={10, 20}, xis=(d1, d2), method="pair")
    p = make(ftq, "ueg_n14_m57", W)
    fd = torch.from_numpy(f).cuda()
    p.propagate(fd[:10].contiguous())
    par1 = p.pair_branch(d1).cpu().numpy()
    p.propagate(fd[10:20].contiguous())
    par2 = p.pair_branch(d2).cpu().numpy()
    p.propagate(fd[20:].contiguous())
    assert np.any(par1 != np.arange(W)) or np.any(par2 != np.arange(W))
    G = p.green().cpu().numpy()
    ws = p.weights().cpu().numpy()
    for w in range(W):
        assert np.abs(G[w] - ref[w].G).max() < 1e-10 * np.abs(ref[w].G).max()
        assert bool(ws[w, 2] > 0.5) == ref[w].alive
        if ref[w].alive:
            assert abs(ws[w, 0] - ref[w].logw.real) < 1e-10 * max(1.0, abs(ref[w].logw.real))
    p.close()
