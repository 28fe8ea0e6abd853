"""Chemical-potential derivative on the GPU against the oracle's central
differences (fixed draws, frozen force bias, h = 1e-4) and closed forms.

Tolerance: the central difference carries an O(h^2) truncation error
(~1e-8 relative here) on top of rounding, so agreement is required to
1e-6 relative for the complex128 path; the mixed path (FP32 chain and
per-slice G) to 1e-4 relative against the complex128 path.
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


def system(wl):
    c = WORKLOADS[wl]
    return dict(N=c["N"], M=c["M"], rs=c["rs"], theta=c["theta"], dtau=c["dtau"])


def test_per_walker_derivatives_match_oracle_fd(ftq):
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 16
    f = gaussian_fields(31, s.n_slices, W, s.N_alpha)
    p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W)
    p.propagate(torch.from_numpy(f).cuda())
    g = p.mu_grad()
    pw = g["per_walker"].cpu().numpy()
    fd = afqmc.mu_derivative_walkers_fd(s, f)
    checked = 0
    for w in range(W):
        if not fd[w]["alive"]:
            continue
        checked += 1
        assert abs(pw[w, 0] - fd[w]["dlogw"]) < 1e-6 * max(1, abs(fd[w]["dlogw"]))
        assert abs(pw[w, 2] - fd[w]["dE"].real) < 1e-6 * max(1, abs(fd[w]["dE"]))
        assert abs(pw[w, 4] - fd[w]["dN"].real) < 1e-6 * max(1, abs(fd[w]["dN"]))
        assert abs(pw[w, 5] - fd[w]["dN"].imag) < 1e-6 * max(1, abs(fd[w]["dN"]))
    assert checked >= W // 2
    ref = afqmc.mu_derivative_fd(s, f)
    assert ref["excluded"] == 0
    assert abs(g["dN"] - ref["dN"]) < 1e-6 * abs(ref["dN"])
    assert abs(g["dE"] - ref["dE"]) < 1e-6 * abs(ref["dE"])


@pytest.mark.timeout(600)
def test_mu_tuning_workload_full_size_sampled_walkers(ftq):
    """The mu-tuning workload at full size (N=14, M=123, r_s=2, Theta=0.25,
    174 slices, 256 walkers, complex128): every walker's d ln|w|/dmu,
    dE_L/dmu and dN_L/dmu from the full launch; three sampled walkers checked
    against the oracle's central differences (h = 1e-4, frozen force bias)."""
    from oracle_pool import walkers_mu_fd
    c = WORKLOADS["ueg_n14_m123"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = c["walkers"]
    f = gaussian_fields(c["seed"], s.n_slices, W, s.N_alpha)
    p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W)
    p.propagate(torch.from_numpy(f).cuda())
    g = p.mu_grad()
    pw = g["per_walker"].cpu().numpy()
    ws = p.weights().cpu().numpy()
    assert p.status() == 0
    p.close()
    alive = [w for w in range(W) if ws[w, 2] > 0.5]
    assert len(alive) >= W // 2
    sample = [alive[0], alive[len(alive) // 2], alive[-1]]
    fd = walkers_mu_fd(system("ueg_n14_m123"), f, sample)
    checked = 0
    for w, r in zip(sample, fd):
        if not r["alive"]:
            continue
        checked += 1
        print(f"walker {w}: dlogw {pw[w, 0]:.10f} / {r['dlogw']:.10f}, dE {pw[w, 2]:.10f} / {r['dE'].real:.10f}, "
              f"dN {pw[w, 4]:.10f} / {r['dN'].real:.10f}")
        assert abs(pw[w, 0] - r["dlogw"]) < 1e-6 * max(1, abs(r["dlogw"]))
        assert abs(pw[w, 2] - r["dE"].real) < 1e-6 * max(1, abs(r["dE"]))
        assert abs(pw[w, 4] - r["dN"].real) < 1e-6 * max(1, abs(r["dN"]))
        assert abs(pw[w, 5] - r["dN"].imag) < 1e-6 * max(1, abs(r["dN"]))
    assert checked >= 2
    assert math.isfinite(g["dN"]) and math.isfinite(g["dE"])


def test_noninteracting_closed_form_full_size(ftq):
    """Zero fields at M=257: the path is free electrons with the propagator's
    energies eps + delta_eps, occupations f, df/dmu = beta f (1 - f):
    d<N>/dmu = 2 sum df and d<E>/dmu = 2 sum eps df - (2/Omega) sum_{K != K'}
    4 pi/|K - K'|^2 f_K df_K' (kinetic plus the exchange term of E_2; the
    Hartree term vanishes for a diagonal P)."""
    c = WORKLOADS["ueg_n66_m257"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 2
    for prec, tol in ((ftq.FTQ_FP64, 1e-9), (ftq.FTQ_MIXED, 2e-5)):
        p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, precision=prec)
        p.propagate(torch.zeros((s.n_slices, W, s.N_alpha), dtype=torch.float64, device="cuda"))
        g = p.mu_grad()
        p.close()
        e = s.eps + s.delta_eps
        ff = fermi_dirac(e, s.mu, s.beta)
        df = s.beta * ff * (1 - ff)
        dn = 2 * np.sum(df)
        kv = s.kvec
        d2 = np.sum((kv[:, None, :] - kv[None, :, :]) ** 2, axis=2)
        np.fill_diagonal(d2, np.inf)
        vkk = 4 * math.pi / d2
        de = 2 * np.sum(s.eps * df) - (2.0 / s.Omega) * (ff @ vkk @ df)
        print(f"precision {prec}: dN {g['dN']:.10f} vs {dn:.10f}; dE {g['dE']:.10f} vs {de:.10f}")
        assert abs(g["dN"] - dn) < tol * dn
        assert abs(g["dE"] - de) < tol * abs(de)


def test_mixed_derivative_matches_complex128(ftq):
    c = WORKLOADS["ueg_n14_m57"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 32
    f = torch.from_numpy(gaussian_fields(77, s.n_slices, W, s.N_alpha)).cuda()
    out = {}
    for prec in (ftq.FTQ_FP64, ftq.FTQ_MIXED):
        p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, precision=prec)
        p.propagate(f)
        out[prec] = p.mu_grad(per_walker=False)
        p.close()
    a, b = out[ftq.FTQ_FP64], out[ftq.FTQ_MIXED]
    print(f"M=57: dN {a['dN']:.8f} / {b['dN']:.8f}, dE {a['dE']:.8f} / {b['dE']:.8f}")
    assert abs(a["dN"] - b["dN"]) < 1e-4 * abs(a["dN"])
    assert abs(a["dE"] - b["dE"]) < 1e-4 * abs(a["dE"])


def test_autograd_and_newton_tuning(ftq):
    """torch.autograd through mu_estimates gives the library derivative; a
    few Newton steps bring <N> to N-bar on fixed fields."""
    sysd = system("ueg_n2_m7")
    s = UEG(sysd["N"], sysd["M"], sysd["rs"], sysd["theta"], sysd["dtau"])
    W = 256
    f = torch.from_numpy(gaussian_fields(5, s.n_slices, W, s.N_alpha)).cuda()
    mu = torch.tensor(s.mu_T, dtype=torch.float64, requires_grad=True)
    out = ftq.mu_estimates(mu, sysd, f, W)
    (gN,) = torch.autograd.grad(out[0], mu)
    p = ftq.Propagator(sysd["N"], sysd["M"], sysd["rs"], sysd["theta"], sysd["dtau"], mu=s.mu_T, walkers=W)
    p.propagate(f)
    ref = p.mu_grad(per_walker=False)
    p.close()
    assert abs(gN.item() - ref["dN"]) < 1e-12 * abs(ref["dN"])
    mu_star, hist = ftq.tune_mu(sysd, f, W, target_n=sysd["N"], mu0=s.mu_T, iterations=4)
    print("Newton history (mu, <N>, d<N>/dmu):", hist)
    assert abs(hist[-1][1] - sysd["N"]) < 1e-6


def test_derivative_requires_full_path(ftq):
    c = WORKLOADS["ueg_n2_m7"]
    p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=2)
    p.propagate(torch.zeros((3, 2, p.n_alpha), dtype=torch.float64, device="cuda"))
    with pytest.raises(ftq.FTQError):
        p.mu_grad()
    p.close()
