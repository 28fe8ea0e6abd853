"""Density correlations <rho(Q) rho(-Q)> (static structure factor) and the
estimators along the imaginary-time path on the GPU against the oracle:
per walker within 1e-10 (complex128), weighted averages, the free-fermion
closed form at the full M = 257, 348-slice scale, and E(tau_k), N(tau_k) at
intermediate slices (the traces and the slice-averaged estimate are these
values at every slice)."""
import math

import numpy as np
import pytest

from oracle import afqmc
from oracle.ueg import UEG, fermi_dirac
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


def oracle_slots(s, G):
    plus, minus = afqmc.density_correlation(s, G)
    out = np.empty(2 * len(plus), np.complex128)
    out[0::2], out[1::2] = plus, minus
    return out


def test_per_walker_and_weighted_match_oracle(ftq):
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 16
    f = gaussian_fields(c["seed"], s.n_slices, W, s.N_alpha)
    ref = afqmc.run(s, f, want_estimator=False)
    p = make(ftq, "ueg_n2_m7", W)
    p.propagate(torch.from_numpy(f).cuda())
    res = p.structure_factor(per_walker=True)
    pw = res["per_walker"].cpu().numpy()
    rows = [oracle_slots(s, r.G) for r in ref]
    for w in range(W):
        assert np.max(np.abs(pw[w] - rows[w])) < 1e-10 * max(1.0, np.max(np.abs(rows[w])))
    lw = np.array([r.logw.real if r.alive else -np.inf for r in ref])
    wt = np.where(np.isfinite(lw), np.exp(lw - lw.max()), 0.0)
    avg = np.sum(wt[:, None] * np.array(rows), axis=0) / wt.sum()
    assert np.max(np.abs(res["rhorho"] - avg)) < 1e-10 * np.max(np.abs(avg))
    q = res["q"]
    assert np.array_equal(q[0::2], np.asarray(s.q_half)) and np.array_equal(q[1::2], -np.asarray(s.q_half))
    assert p.status() == 0
    p.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 2e-5)])
def test_free_fermion_closed_form_full_size(ftq, prec, tol):
    """Zero fields at M = 257: G(beta) = diag(1 - f) with the propagator's
    energies, so <rho(Q) rho(-Q)> = 2 sum_K f_{K+Q} (1 - f_K)."""
    c = WORKLOADS["ueg_n66_m257"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 2
    p = make(ftq, "ueg_n66_m257", W, precision=ftq.FTQ_FP64 if prec == "fp64" else ftq.FTQ_MIXED)
    p.propagate(torch.zeros((s.n_slices, W, s.N_alpha), dtype=torch.float64, device="cuda"))
    res = p.structure_factor()
    p.close()
    fk = fermi_dirac(s.eps + s.delta_eps, s.mu, s.beta)
    index = {tuple(v): i for i, v in enumerate(s.nvec)}
    for j, qv in enumerate(res["q"]):
        ref = 0.0
        for k in range(s.M):
            kq = index.get(tuple(s.nvec[k] + qv))
            if kq is not None:
                ref += 2.0 * fk[kq] * (1.0 - fk[k])
        assert abs(res["rhorho"][j] - ref) < tol * max(1.0, ref), (j, qv, res["rhorho"][j], ref)
    assert np.allclose(res["S"], res["rhorho"].real / c["N"])


def test_estimators_along_the_path_match_oracle(ftq):
    """E(tau_k), N(tau_k) per walker at intermediate slices from G(tau_k)."""
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 8
    f = gaussian_fields(c["seed"], s.n_slices, W, s.N_alpha)
    fd = torch.from_numpy(f).cuda()
    p = make(ftq, "ueg_n2_m7", W)
    done = 0
    for k in (5, 11, 17):
        p.propagate(fd[done:k].contiguous())
        done = k
        est = p.estimators(per_walker=True)["per_walker"].cpu().numpy()
        ref = afqmc.run(s, f[:k], n_slices=k, want_estimator=False)
        for w in range(W):
            E, Nn = afqmc.local_energy(s, ref[w].G)
            assert abs(est[w, 3] - E.real) < 1e-10 * max(1.0, abs(E))
            assert abs(est[w, 5] - Nn.real) < 1e-10 * max(1.0, abs(Nn))
    p.close()


def test_mixed_matches_fp64(ftq):
    c = WORKLOADS["ueg_n14_m57"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 8
    fd = torch.from_numpy(gaussian_fields(c["seed"], 20, W, s.N_alpha)).cuda()
    out = {}
    for prec in (ftq.FTQ_FP64, ftq.FTQ_MIXED):
        p = make(ftq, "ueg_n14_m57", W, precision=prec)
        p.propagate(fd)
        out[prec] = p.structure_factor()["rhorho"]
        p.close()
    a, b = out[ftq.FTQ_FP64], out[ftq.FTQ_MIXED]
    assert np.max(np.abs(a - b)) < 1e-5 * np.max(np.abs(a))
