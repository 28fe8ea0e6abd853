"""Time-slice estimates and their average (ftq_track_estimates /
ftq_slice_estimates; Results, "Assessing the Phaseless Constraint": "No
Average" vs "Average") against the oracle's slice_estimates on identical
fields, and, without a constraint, against the exact mixed estimates of
Fock-space diagonalisation.

Tolerances: 1e-10 relative for the complex128 path (the estimators round
in a different order from the oracle); the mixed path's slice estimates use
the FP32 G(tau_k) of each slice and are held to the 1e-5 Ha/e bar of the
mixed precision form against the complex128 path."""
import math

import numpy as np
import pytest

from oracle import afqmc, ed
from oracle.ueg import UEG
from synthetic_inputs import WORKLOADS, gaussian_fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
RTOL = 1e-10


@pytest.fixture(scope="module")
def ftq():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2012_12228_gb300 as m
    return m


def make(ftq, wl, W, **kw):
    c = WORKLOADS[wl]
    return ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, **kw)


@pytest.mark.parametrize("every", [1, 5])
def test_slice_estimates_match_oracle_config1(ftq, every):
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 64
    f = gaussian_fields(c["seed"], s.n_slices, W, s.N_alpha)
    p = make(ftq, "ueg_n2_m7", W)
    p.track_estimates(every)
    fd = torch.from_numpy(f).cuda()
    p.propagate(fd[:9].contiguous())            # two calls: the record continues across them
    p.propagate(fd[9:].contiguous())
    got = p.slice_estimates()
    ks, Ek, Nk, Ea, Na = afqmc.slice_estimates(s, f, every=every)
    assert list(got["k"]) == ks
    assert np.max(np.abs(got["E"] - Ek) / np.abs(Ek)) < RTOL
    assert np.max(np.abs(got["N"] - Nk) / np.abs(Nk)) < RTOL
    assert abs(got["E_avg"].real - Ea) < RTOL * abs(Ea)
    assert abs(got["N_avg"].real - Na) < RTOL * abs(Na)
    # a record at tau = beta is the estimate of ftq_estimators
    est = p.estimators()
    if ks[-1] == s.n_slices:
        assert abs(got["E"][-1] - est["E"]) < RTOL * abs(est["E"])
    p.reset()
    p.propagate(fd[:3].contiguous())
    assert len(p.slice_estimates()["k"]) == 3 // every
    assert p.status() == 0
    p.close()


def test_free_projection_slice_estimates_match_exact_mixed_estimates(ftq):
    """No constraint, 8 x 2048 walkers: at every slice the GPU estimate is
    within 3 standard errors (over the 8 groups) plus the Trotter allowance
    of the exact tr(e^{-k dtau (H - mu N)} B_T^(n-k) O) / tr(...) estimate."""
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    n = s.n_slices
    groups, W = 8, 2048
    E = np.zeros((groups, n))
    N = np.zeros((groups, n))
    for g in range(groups):
        p = make(ftq, "ueg_n2_m7", W, constraint=ftq.FTQ_FREE)
        p.track_estimates(1)
        p.propagate(torch.from_numpy(gaussian_fields(4000 + g, n, W, s.N_alpha)).cuda())
        r = p.slice_estimates()
        E[g], N[g] = r["E"].real, r["N"].real
        p.close()
    exact = [ed.mixed_estimate(s, k * s.dtau, (n - k) * s.dtau) for k in range(1, n + 1)]
    for k in range(n):
        eE = E[:, k].std(ddof=1) / math.sqrt(groups)
        eN = N[:, k].std(ddof=1) / math.sqrt(groups)
        assert abs(E[:, k].mean() - exact[k][0].real) < 3 * eE + 5e-3, (k + 1, E[:, k].mean(), eE, exact[k][0])
        assert abs(N[:, k].mean() - exact[k][1].real) < 3 * eN + 2e-3, (k + 1, N[:, k].mean(), eN, exact[k][1])


def test_mixed_slice_estimates_vs_complex128_config2(ftq):
    """N=14, M=57, 64 walkers, every slice of the 87-slice path: the mixed
    path's slice estimates (FP32 G of each slice) within 1e-5 Ha/e and 1e-5
    electrons of the complex128 path's, and so is the slice average."""
    c = WORKLOADS["ueg_n14_m57"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 64
    f = torch.from_numpy(gaussian_fields(c["seed"], s.n_slices, W, s.N_alpha)).cuda()
    out = {}
    for prec in (ftq.FTQ_FP64, ftq.FTQ_MIXED):
        p = make(ftq, "ueg_n14_m57", W, precision=prec)
        p.track_estimates(1)
        p.propagate(f)
        out[prec] = p.slice_estimates()
        assert p.status() == 0
        p.close()
    a, b = out[ftq.FTQ_FP64], out[ftq.FTQ_MIXED]
    dE = np.max(np.abs(a["E"].real - b["E"].real)) / c["N"]
    dN = np.max(np.abs(a["N"].real - b["N"].real))
    print(f"M=57 slice estimates, mixed vs complex128: max |dE_k|/N {dE:.2e} Ha, max |dN_k| {dN:.2e}; "
          f"averages E/N {a['E_avg'].real / c['N']:.8f} vs {b['E_avg'].real / c['N']:.8f}")
    assert dE < 1e-5 and dN < 1e-5
    assert abs(a["E_avg"].real - b["E_avg"].real) / c["N"] < 1e-5


def test_slice_estimates_config2_vs_oracle(ftq):
    """complex128, N=14, M=57, 12 walkers, slices 29, 58 and 87 against the
    oracle's slice estimates."""
    c = WORKLOADS["ueg_n14_m57"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 12
    f = gaussian_fields(c["seed"] + 5, s.n_slices, W, s.N_alpha)
    p = make(ftq, "ueg_n14_m57", W)
    p.track_estimates(29)
    p.propagate(torch.from_numpy(f).cuda())
    got = p.slice_estimates()
    p.close()
    ks, Ek, Nk, Ea, Na = afqmc.slice_estimates(s, f, every=29)
    assert list(got["k"]) == ks == [29, 58, 87]
    assert np.max(np.abs(got["E"] - Ek) / np.abs(Ek)) < RTOL
    assert np.max(np.abs(got["N"] - Nk) / np.abs(Nk)) < RTOL


def test_tracking_arguments(ftq):
    p = make(ftq, "ueg_n2_m7", 2)
    with pytest.raises(ftq.FTQError):
        p.slice_estimates()                     # never enabled
    with pytest.raises(ftq.FTQError):
        p.track_estimates(-1)
    p.track_estimates(0)
    p.close()
