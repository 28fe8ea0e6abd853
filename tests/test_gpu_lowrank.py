"""Low-rank truncation on the GPU (opts.low_rank_threshold) against the
oracle (Options(low_rank=thr)).

complex128: the same rank of every walker at every stabilisation (exact),
G, ln det, ln|w| and per-walker estimators within 1e-10 (measured ~1e-14,
printed); with a threshold below
every scale it equals the full-rank GPU path; at the full 348-slice M = 257
scale and the paper's threshold 1e-6 it agrees with full rank within 1e-5
while the rank drops.

Mixed (tensor-core chain on the kept columns only, the truncated QR and the
Woodbury Green's function in complex128 on a copy of the chain): the same
ranks as the oracle when no truncation decision lies within 1e-5 relative
of the threshold (the FP32 chain moves |R_jj| by ~1e-6 relative), G within
1e-4, ln det within 1e-5 relative, the local energies within 1e-5
relative; against the complex128 low-rank path at the full M = 257 scale."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import afqmc
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


def oracle_with_margins(s, f, thr, n=None):
    """Oracle paths with low rank, and the smallest relative distance of a
    truncation decision (|R_jj| or a trial-block entry) to the threshold."""
    margins = []
    orig = afqmc.stabilise_truncated

    def recording(Y, D, T, t):
        _, R, _ = sla.qr(Y * D[None, :], pivoting=True, mode="economic")
        margins.append(np.min(np.abs(np.abs(np.diag(R)) / t - 1.0)))
        return orig(Y, D, T, t)

    afqmc.stabilise_truncated = recording
    try:
        ref = afqmc.run(s, f, afqmc.Options(low_rank=thr), n_slices=n, record=True)
    finally:
        afqmc.stabilise_truncated = orig
    for k in range(0, (n or s.n_slices) + 1):
        margins.append(np.min(np.abs(afqmc.left_diagonal(s, k) / thr - 1.0)))
    return ref, min(margins)


def test_matches_oracle_with_truncation(ftq):
    c = WORKLOADS["ueg_n14_m57"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W, thr = 8, 1e-3
    f = gaussian_fields(c["seed"] + 60, s.n_slices, W, s.N_alpha)
    ref, margin = oracle_with_margins(s, f, thr)
    assert margin > 1e-8
    p = make(ftq, "ueg_n14_m57", W, low_rank=thr)
    fd = torch.from_numpy(f).cuda()
    for k0 in range(0, s.n_slices, 29):
        k1 = min(k0 + 29, s.n_slices)
        p.propagate(fd[k0:k1].contiguous())
        ranks = p.ranks()
        assert [r.rank_trace[k1 - 1] for r in ref] == list(ranks), (k1, ranks)
    assert min(r.rank_trace[-1] for r in ref) < s.M          # the rank dropped
    G = p.green().cpu().numpy()
    ws = p.weights().cpu().numpy()
    est = p.estimators(per_walker=True)["per_walker"].cpu().numpy()
    eg = el = ed = ee = 0.0
    for w in range(W):
        r = ref[w]
        eg = max(eg, np.abs(G[w] - r.G).max() / np.abs(r.G).max())
        ed = max(ed, abs(ws[w, 3] - r.logdet.real) / max(1.0, abs(r.logdet.real)))
        assert bool(ws[w, 2] > 0.5) == r.alive
        if r.alive:
            el = max(el, abs(ws[w, 0] - r.logw.real) / max(1.0, abs(r.logw.real)))
            ee = max(ee, abs(est[w, 3] - r.energy.real) / max(1.0, abs(r.energy)))
            assert abs(est[w, 5] - r.number.real) < 1e-10 * max(1.0, abs(r.number))
    print(f"low rank complex128 vs oracle, M=57 whole path: G {eg:.1e}, ln det {ed:.1e}, ln|w| {el:.1e}, E_L {ee:.1e}")
    assert eg < 1e-10 and ed < 1e-10
    assert el < 1e-10 and ee < 1e-10
    assert p.status() == 0
    p.close()


def test_mixed_matches_oracle_with_truncation(ftq):
    c = WORKLOADS["ueg_n14_m57"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W, thr = 8, 1e-3
    f = gaussian_fields(c["seed"] + 60, s.n_slices, W, s.N_alpha)
    ref, margin = oracle_with_margins(s, f, thr)
    assert margin > 1e-5
    p = make(ftq, "ueg_n14_m57", W, low_rank=thr, precision=ftq.FTQ_MIXED)
    fd = torch.from_numpy(f).cuda()
    for k0 in range(0, s.n_slices, 29):
        k1 = min(k0 + 29, s.n_slices)
        p.propagate(fd[k0:k1].contiguous())
        ranks = p.ranks()
        assert [r.rank_trace[k1 - 1] for r in ref] == list(ranks), (k1, ranks)
    assert min(r.rank_trace[-1] for r in ref) < s.M
    G = p.green().cpu().numpy()
    ws = p.weights().cpu().numpy()
    est = p.estimators(per_walker=True)["per_walker"].cpu().numpy()
    eg = ed = ee = 0.0
    for w in range(W):
        r = ref[w]
        eg = max(eg, np.abs(G[w] - r.G).max() / np.abs(r.G).max())
        ed = max(ed, abs(ws[w, 3] - r.logdet.real) / max(1.0, abs(r.logdet.real)))
        assert bool(ws[w, 2] > 0.5) == r.alive
        if r.alive:
            ee = max(ee, abs(est[w, 3] - r.energy.real) / max(1.0, abs(r.energy)))
            assert abs(ws[w, 0] - r.logw.real) < 2e-5 * max(1.0, abs(r.logdet.real))
    print(f"low rank mixed vs oracle, M=57 whole path: G {eg:.1e}, ln det {ed:.1e}, E_L {ee:.1e}")
    assert eg < 1e-4 and ed < 1e-5 and ee < 1e-5
    assert p.status() == 0
    p.close()


def test_mixed_low_rank_full_size(ftq):
    """N = 66, M = 257, the whole 348-slice path, 2 walkers, threshold 1e-6:
    the mixed low-rank path against the complex128 low-rank path."""
    c = WORKLOADS["ueg_n66_m257"]
    W = 2
    fd = torch.from_numpy(gaussian_fields(c["seed"] + 62, 348, W, 1796)).cuda()
    res = []
    for prec in (ftq.FTQ_FP64, ftq.FTQ_MIXED):
        p = make(ftq, "ueg_n66_m257", W, low_rank=1e-6, precision=prec)
        p.propagate(fd)
        e = p.estimators(per_walker=True)["per_walker"].cpu().numpy()
        res.append((e, p.weights().cpu().numpy(), p.ranks()))
        assert p.status() == 0
        p.close()
    (ea, wa, ra), (eb, wb, rb) = res
    print(f"M=257 low rank, ranks complex128 {list(ra)} mixed {list(rb)}")
    assert np.all(rb < 0.7 * 257)
    assert np.all(np.abs(ra - rb) <= 2)
    alive = (wa[:, 2] > 0.5) & (wb[:, 2] > 0.5)
    assert alive.any()
    dE = np.max(np.abs(ea[alive, 3] - eb[alive, 3])) / 66
    print(f"M=257 low rank, mixed vs complex128: |dE_L|/N {dE:.1e} Ha")
    assert dE < 1e-5
    assert np.max(np.abs(ea[alive, 5] - eb[alive, 5])) < 1e-5 * 66


def test_untruncated_equals_full_rank_gpu(ftq):
    c = WORKLOADS["ueg_n14_m57"]
    W = 8
    fd = torch.from_numpy(gaussian_fields(c["seed"] + 61, 22, W, 340)).cuda()
    out = []
    for thr in (0.0, 1e-300):
        p = make(ftq, "ueg_n14_m57", W, low_rank=thr)
        p.propagate(fd)
        out.append((p.green().cpu().numpy(), p.weights().cpu().numpy(), p.ranks()))
        p.close()
    (Ga, wa, ra), (Gb, wb, rb) = out
    assert np.all(ra == 57) and np.all(rb == 57)
    assert np.abs(Ga - Gb).max() < 1e-10 * np.abs(Ga).max()
    assert np.max(np.abs(wa[:, 0] - wb[:, 0])) < 1e-10 * max(1.0, np.max(np.abs(wa[:, 0])))


def test_full_size_paper_threshold(ftq):
    """N = 66, M = 257, Theta = 0.0625, the whole 348-slice path, 2 walkers."""
    c = WORKLOADS["ueg_n66_m257"]
    W = 2
    fd = torch.from_numpy(gaussian_fields(c["seed"] + 62, 348, W, 1796)).cuda()
    res = []
    for thr in (0.0, 1e-6):
        p = make(ftq, "ueg_n66_m257", W, low_rank=thr)
        p.propagate(fd)
        e = p.estimators(per_walker=True)["per_walker"].cpu().numpy()
        res.append((e, p.weights().cpu().numpy(), p.ranks()))
        assert p.status() == 0
        p.close()
    (ea, wa, ra), (eb, wb, rb) = res
    assert np.all(ra == 257) and np.all(rb < 0.7 * 257)
    alive = (wa[:, 2] > 0.5) & (wb[:, 2] > 0.5)
    assert alive.any()
    assert np.max(np.abs(ea[alive, 3] - eb[alive, 3])) < 1e-5 * np.max(np.abs(ea[alive, 3]))
    assert np.max(np.abs(ea[alive, 5] - eb[alive, 5])) < 1e-5 * 66


def test_rejected_arguments(ftq):
    with pytest.raises(ftq.FTQError):
        make(ftq, "ueg_n2_m7", 4, precision=ftq.FTQ_MIXED_SIMT, low_rank=1e-6)
    with pytest.raises(ftq.FTQError):
        make(ftq, "ueg_n2_m7", 4, low_rank=-1.0)


def test_mu_derivative_with_low_rank(ftq):
    """Per-walker mu derivatives along a truncated path (the trial block
    keeps fewer than its 7 entries early on) against the oracle's central
    differences."""
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W, thr = 16, 0.05
    assert np.sum(afqmc.left_diagonal(s, 1) >= thr) < s.M
    f = gaussian_fields(c["seed"] + 63, s.n_slices, W, s.N_alpha)
    p = make(ftq, "ueg_n2_m7", W, low_rank=thr)
    p.propagate(torch.from_numpy(f).cuda())
    pw = p.mu_grad()["per_walker"].cpu().numpy()
    p.close()
    fd = afqmc.mu_derivative_walkers_fd(s, f, afqmc.Options(low_rank=thr))
    checked = 0
    for w in range(W):
        if not fd[w]["alive"]:
            continue
        checked += 1
        assert abs(pw[w, 0] - fd[w]["dlogw"]) < 1e-6 * max(1, abs(fd[w]["dlogw"]))
        assert abs(pw[w, 2] - fd[w]["dE"].real) < 1e-6 * max(1, abs(fd[w]["dE"]))
        assert abs(pw[w, 4] - fd[w]["dN"].real) < 1e-6 * max(1, abs(fd[w]["dN"]))
    assert checked >= W // 2


def test_population_control_with_low_rank(ftq):
    """Combs between truncated slices copy the whole walker state, rank
    included: the path equals the oracle's comb path."""
    from oracle.population import run_with_population_control
    c = WORKLOADS["ueg_n14_m57"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W, thr = 16, 1e-3
    f = gaussian_fields(c["seed"] + 64, s.n_slices, W, s.N_alpha)
    ref = run_with_population_control(s, f, pc_after={40, 60}, xis=(0.3, 0.71), opts=afqmc.Options(low_rank=thr))
    p = make(ftq, "ueg_n14_m57", W, low_rank=thr)
    fd = torch.from_numpy(f).cuda()
    p.propagate(fd[:40].contiguous())
    p.population_control(0.3)
    p.propagate(fd[40:60].contiguous())
    p.population_control(0.71)
    p.propagate(fd[60:].contiguous())
    G = p.green().cpu().numpy()
    ws = p.weights().cpu().numpy()
    assert list(p.ranks()) == [len(r.D) for r in ref]
    for w in range(W):
        assert np.abs(G[w] - ref[w].G).max() < 1e-10 * np.abs(ref[w].G).max()
        assert bool(ws[w, 2] > 0.5) == ref[w].alive
        if ref[w].alive:
            assert abs(ws[w, 0] - ref[w].logw.real) < 1e-10 * max(1.0, abs(ref[w].logw.real))
    assert p.status() == 0
    p.close()
