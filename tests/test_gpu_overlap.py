"""The modified overlap ratio (Eq. ztfix, FTQ_OVERLAP_MODIFIED) on the GPU
against the oracle (Options(overlap="modified")): G(tau_k) of A~_k = B_T^n
B_k ... B_1 at intermediate slices, and at tau = beta the physical G(beta),
the weights after the final ratio and the per-walker estimators, within
1e-10 in complex128 (phaseless and free projection); the mixed path against
complex128 within 1e-5."""
import math

import numpy as np
import pytest

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
    return ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W,
                          overlap=ftq.FTQ_OVERLAP_MODIFIED, **kw)


def wrap(a):
    return np.remainder(a + np.pi, 2 * np.pi) - np.pi


@pytest.mark.parametrize("constraint", ["phaseless", "free"])
def test_full_path_matches_oracle(ftq, constraint):
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 16
    f = gaussian_fields(c["seed"] + 40, s.n_slices, W, s.N_alpha)
    ref = afqmc.run(s, f, afqmc.Options(constraint=constraint, overlap="modified"))
    p = make(ftq, "ueg_n2_m7", W, constraint=ftq.FTQ_FREE if constraint == "free" else ftq.FTQ_PHASELESS)
    p.propagate(torch.from_numpy(f).cuda())
    G = p.green().cpu().numpy()
    ws = p.weights().cpu().numpy()
    est = p.estimators(per_walker=True)["per_walker"].cpu().numpy()
    for w in range(W):
        r = ref[w]
        assert np.abs(G[w] - r.G).max() < 1e-10 * np.abs(r.G).max()
        assert bool(ws[w, 2] > 0.5) == r.alive
        if r.alive:
            assert abs(ws[w, 0] - r.logw.real) < 1e-9 * max(1.0, abs(r.logw.real))
            assert abs(est[w, 3] - r.energy.real) < 1e-10 * max(1.0, abs(r.energy))
            assert abs(est[w, 5] - r.number.real) < 1e-10 * max(1.0, abs(r.number))
        if constraint == "free":
            assert abs(wrap(ws[w, 1] - r.logw.imag)) < 1e-9
    assert p.status() == 0
    p.close()


def test_intermediate_slices_use_the_full_trial_block(ftq):
    """Before slice n the library's G is that of A~_k = B_T^n B_k ... B_1."""
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W, k = 8, 13
    f = gaussian_fields(c["seed"] + 41, s.n_slices, W, s.N_alpha)
    ref = afqmc.run(s, f[:k], afqmc.Options(overlap="modified"), n_slices=k, want_estimator=False)
    p = make(ftq, "ueg_n2_m7", W)
    p.propagate(torch.from_numpy(f[:k].copy()).cuda())
    G = p.green().cpu().numpy()
    ws = p.weights().cpu().numpy()
    for w in range(W):
        assert np.abs(G[w] - ref[w].G).max() < 1e-10 * np.abs(ref[w].G).max()
        assert bool(ws[w, 2] > 0.5) == ref[w].alive
        if ref[w].alive:
            assert abs(ws[w, 0] - ref[w].logw.real) < 1e-9 * max(1.0, abs(ref[w].logw.real))
    p.close()


def test_mixed_matches_fp64(ftq):
    c = WORKLOADS["ueg_n14_m57"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 8
    fd = torch.from_numpy(gaussian_fields(c["seed"] + 42, s.n_slices, W, s.N_alpha)).cuda()
    out = {}
    for prec in (ftq.FTQ_FP64, ftq.FTQ_MIXED):
        p = make(ftq, "ueg_n14_m57", W, precision=prec)
        p.propagate(fd)
        out[prec] = (p.green().cpu().numpy(), p.weights().cpu().numpy(),
                     p.estimators(per_walker=True)["per_walker"].cpu().numpy())
        assert p.status() == 0
        p.close()
    (Ga, wa, ea), (Gb, wb, eb) = out[ftq.FTQ_FP64], out[ftq.FTQ_MIXED]
    alive = (wa[:, 2] > 0.5) & (wb[:, 2] > 0.5)
    assert alive.sum() >= W // 2
    assert np.abs(Ga[alive] - Gb[alive]).max() < 1e-5 * np.abs(Ga).max()
    # ln|w| telescopes to 2 ln det: twice the 1e-5 relative bound of the FP32 ln det
    assert np.max(np.abs(wa[alive, 0] - wb[alive, 0])) < 2e-5 * max(1.0, np.max(np.abs(wa[alive, 3])))
    assert np.max(np.abs(ea[alive, 3] - eb[alive, 3])) < 1e-5 * np.max(np.abs(ea[alive, 3]))


def test_mu_derivative_with_modified_overlap(ftq):
    """d ln|w|/dmu, dE_L/dmu, dN_L/dmu per walker (fixed draws, frozen force
    bias) against the oracle's central differences along the modified path,
    the final ratio r included."""
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 16
    f = gaussian_fields(c["seed"] + 43, s.n_slices, W, s.N_alpha)
    p = make(ftq, "ueg_n2_m7", W)
    p.propagate(torch.from_numpy(f).cuda())
    pw = p.mu_grad()["per_walker"].cpu().numpy()
    p.close()
    fd = afqmc.mu_derivative_walkers_fd(s, f, afqmc.Options(overlap="modified"))
    checked = 0
    for w in range(W):
        if not fd[w]["alive"]:
            continue
        checked += 1
        assert abs(pw[w, 0] - fd[w]["dlogw"]) < 1e-6 * max(1, abs(fd[w]["dlogw"]))
        assert abs(pw[w, 2] - fd[w]["dE"].real) < 1e-6 * max(1, abs(fd[w]["dE"]))
        assert abs(pw[w, 4] - fd[w]["dN"].real) < 1e-6 * max(1, abs(fd[w]["dN"]))
    assert checked >= W // 2
