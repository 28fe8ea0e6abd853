"""Mixed-precision path (FP32 chain in tf32 hi/lo planes, FP32 G(tau) per
slice, complex128 QRCP, complex128 G(beta), FP64 log-weights) against the
oracle and the complex128 GPU path on identical fields.

Tolerances are stated from the arithmetic: the chain stores values as
hi + lo tf32 pairs (relative error <= 2^-22 = 2.4e-7 per rounding) and the
per-slice LU runs in FP32 (unit roundoff 6e-8 times the growth of a
well-conditioned, pivoted M x M system); a path of n slices accumulates
these, so G(beta) is held to 1e-4 relative and the weighted energy per
electron to the mixed-precision accuracy bound of 1e-5 Ha.
"""
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


def make(ftq, wl, W, precision, **kw):
    p = WORKLOADS[wl]
    return ftq.Propagator(p["N"], p["M"], p["rs"], p["theta"], p["dtau"], walkers=W, precision=precision, **kw)


def weighted_e_per_electron(est, N):
    return est["E"].real / N


@pytest.mark.parametrize("wl,W,n", [("ueg_n2_m7", 16, 3), ("ueg_n14_m57", 8, 6), ("ueg_n14_m123", 4, 6),
                                    ("ueg_n66_m257", 4, 6)])
def test_tensor_chain_matches_cuda_core_chain(ftq, wl, W, n):
    """tcgen05 3xTF32 chain vs the FP32 CUDA-core chain on the same fields:
    both hold the chain to ~2^-22; they differ by the dropped lo*lo product
    and the summation order, so G agrees to ~1e-6 after a QRCP block."""
    c = WORKLOADS[wl]
    f = torch.from_numpy(gaussian_fields(c["seed"], n, W, UEG(c["N"], c["M"], c["rs"], c["theta"],
                                                               c["dtau"]).N_alpha)).cuda()
    out = {}
    for prec in (ftq.FTQ_MIXED_SIMT, ftq.FTQ_MIXED):
        p = make(ftq, wl, W, prec)
        p.propagate(f)
        out[prec] = (p.green().cpu().numpy(), p.weights().cpu().numpy())
        assert p.status() == 0
        p.close()
    ga, gb = out[ftq.FTQ_MIXED_SIMT][0], out[ftq.FTQ_MIXED][0]
    err = np.abs(ga - gb).max() / np.abs(ga).max()
    lerr = np.abs(out[ftq.FTQ_MIXED_SIMT][1][:, 3] - out[ftq.FTQ_MIXED][1][:, 3]).max()
    print(f"{wl}: tensor vs CUDA-core chain, G rel err {err:.2e}, ln det abs err {lerr:.2e}")
    assert err < 1e-5
    assert lerr < 1e-4


@pytest.mark.parametrize("prec", ["mixed", "mixed_simt"])
def test_mixed_vs_oracle_config1(ftq, prec):
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 32
    f = gaussian_fields(c["seed"], s.n_slices, W, s.N_alpha)
    p = make(ftq, "ueg_n2_m7", W, ftq.FTQ_MIXED if prec == "mixed" else ftq.FTQ_MIXED_SIMT)
    fd = torch.from_numpy(f).cuda()
    p.propagate(fd[:10].contiguous())
    G10 = p.green().cpu().numpy()
    p.propagate(fd[10:].contiguous())
    G = p.green().cpu().numpy()
    ws = p.weights().cpu().numpy()
    ref = afqmc.run(s, f)
    ref10 = afqmc.run(s, f[:10], n_slices=10, want_estimator=False)
    errs = []
    for w in range(W):
        errs.append(np.abs(G[w] - ref[w].G).max() / np.abs(ref[w].G).max())
        assert np.abs(G10[w] - ref10[w].G).max() < 1e-5
        assert (ws[w, 2] > 0.5) == ref[w].alive
        if ref[w].alive:
            # ln|w| telescopes to 2 ln det: twice the 1e-5 relative bound of the FP32 ln det
            assert abs(ws[w, 0] - ref[w].logw.real) < 2e-5 * max(1, abs(ref[w].logdet.real))
    print(f"mixed vs oracle, M=7: max rel err G(beta) {max(errs):.2e}")
    assert max(errs) < 1e-4


def test_mixed_vs_fp64_energy_config2(ftq):
    """N=14, M=57, whole path: |E/N (mixed) - E/N (complex128)| <= 1e-5 Ha."""
    c = WORKLOADS["ueg_n14_m57"]
    W = 64
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    f = torch.from_numpy(gaussian_fields(c["seed"], s.n_slices, W, s.N_alpha)).cuda()
    res = {}
    for prec in (ftq.FTQ_FP64, ftq.FTQ_MIXED):
        p = make(ftq, "ueg_n14_m57", W, prec)
        p.propagate(f)
        est = p.estimators()
        res[prec] = (est, p.green().cpu().numpy(), p.weights().cpu().numpy())
        assert p.status() == 0
        p.close()
    e64 = weighted_e_per_electron(res[ftq.FTQ_FP64][0], c["N"])
    e32 = weighted_e_per_electron(res[ftq.FTQ_MIXED][0], c["N"])
    gerr = max(np.abs(a - b).max() / np.abs(a).max() for a, b in zip(res[ftq.FTQ_FP64][1], res[ftq.FTQ_MIXED][1]))
    alive64 = res[ftq.FTQ_FP64][2][:, 2] > 0.5
    alive32 = res[ftq.FTQ_MIXED][2][:, 2] > 0.5
    print(f"M=57 n=87: E/N fp64 {e64:.10f} mixed {e32:.10f} diff {abs(e64 - e32):.2e}; max rel G err {gerr:.2e}")
    assert np.array_equal(alive64, alive32)
    assert abs(e64 - e32) <= 1e-5
    assert gerr < 1e-4


def test_mixed_noninteracting_full_size(ftq):
    """Zero fields at M=257, beta=8.69, 348 slices: G(beta) = diag(1 - f_FD)
    and 2 ln det = ln Z_0 through the FP32 chain and FP32 per-slice LU."""
    c = WORKLOADS["ueg_n66_m257"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 2
    p = make(ftq, "ueg_n66_m257", W, ftq.FTQ_MIXED)
    p.propagate(torch.zeros((s.n_slices, W, s.N_alpha), dtype=torch.float64, device="cuda"))
    G = p.green().cpu().numpy()
    ws = p.weights().cpu().numpy()
    e = s.eps + s.delta_eps
    fd = fermi_dirac(e, s.mu, s.beta)
    ld = np.sum(np.log1p(np.exp(-s.beta * (e - s.mu))))
    for w in range(W):
        err = np.abs(G[w] - np.diag(1 - fd)).max()
        print(f"mixed non-interacting M=257: G err {err:.2e}, ln det rel err {abs(ws[w, 3] - ld) / ld:.2e}")
        # per orbital ln d drifts by <= n * 2^-22 = 8.3e-5 (tf32 hi/lo storage,
        # one rounding per slice); G = 1 - f moves by f(1-f) times that
        assert err < 3e-5
        assert abs(ws[w, 3] - ld) < 1e-5 * ld
