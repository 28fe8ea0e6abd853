"""CUDA path vs the CPU oracle on identical seeded fields (complex128).

Tolerance: 1e-10 relative on G(tau), ln|w| and ln det(I + A), element by
element, as the complex128 path must reach (rounding differs only in the
order of operations and in the QRCP / LU pivot sequence; G and the
determinants do not depend on either).  Phaseless kills (cos theta <= 0)
must agree walker by walker.
"""
import math

import numpy as np
import pytest

from oracle import afqmc, ed
from oracle.ueg import UEG, fermi_dirac
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


def make(ftq, wl, W=None, **kw):
    p = dict(WORKLOADS[wl])
    return ftq.Propagator(p["N"], p["M"], p["rs"], p["theta"], p["dtau"], walkers=W or p["walkers"], **kw)


def oracle_states(sys, fields, opts, n, walkers):
    """Oracle state of each walker in `walkers` after every slice 1..n."""
    out = []
    for w in walkers:
        st = afqmc.initial_state(sys)
        trace = []
        for k in range(1, n + 1):
            st, *_ = afqmc.slice_step(sys, st, fields[k - 1, w], k, opts)
            trace.append(st)
        out.append(trace)
    return out


def assert_walker_close(G_gpu, ws_gpu, st, where):
    scale = max(np.abs(st.G).max(), 1e-300)
    err = np.abs(G_gpu - st.G).max() / scale
    assert err < RTOL, f"{where}: G rel err {err:.3e}"
    assert bool(ws_gpu[2] > 0.5) == bool(st.alive), f"{where}: alive flag differs"
    if st.alive:
        lw = st.logw.real
        assert abs(ws_gpu[0] - lw) < RTOL * max(1.0, abs(lw)), f"{where}: ln|w| {ws_gpu[0]} vs {lw}"
    ld = st.logdet
    assert abs(ws_gpu[3] - ld.real) < RTOL * max(1.0, abs(ld.real)), f"{where}: ln det"
    assert abs(math.remainder(ws_gpu[4] - ld.imag, 2 * math.pi)) < 1e-9, f"{where}: arg det"


def test_conventions_match_oracle(ftq):
    """Basis order, half-space transfers, beta, dtau, mu_T and E_M agree."""
    for wl in ("ueg_n2_m7", "ueg_n14_m57", "ueg_n66_m257"):
        p = make(ftq, wl, W=1)
        c = WORKLOADS[wl]
        s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
        assert p.basis() == [tuple(int(x) for x in n) for n in s.nvec]
        assert p.transfers() == [tuple(int(x) for x in q) for q in s.q_half]
        assert p.n_slices == s.n_slices and p.n_alpha == s.N_alpha
        for key, ref in (("BETA", s.beta), ("DTAU", s.dtau), ("MU_T", s.mu_T), ("E_M", s.E_M), ("L", s.L)):
            assert abs(p.query_f64(key) - ref) < 1e-12 * max(1.0, abs(ref)), key
        p.close()


def test_parity_config1_every_slice(ftq):
    """N=2, M=7, 64 walkers, the whole path (22 slices, QRCP every 5)."""
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = c["walkers"]
    f = gaussian_fields(c["seed"], s.n_slices, W, s.N_alpha)
    p = make(ftq, "ueg_n2_m7")
    ref = oracle_states(s, f, afqmc.Options(), s.n_slices, range(W))
    fd = torch.from_numpy(f).cuda()
    for k in range(1, s.n_slices + 1):
        p.propagate(fd[k - 1:k].contiguous())
        G = p.green().cpu().numpy()
        ws = p.weights().cpu().numpy()
        for w in range(W):
            assert_walker_close(G[w], ws[w], ref[w][k - 1], f"slice {k} walker {w}")
    est = p.estimators()
    pw = est["per_walker"].cpu().numpy()
    for w in range(W):
        E, Nn = afqmc.local_energy(s, ref[w][-1].G)
        assert abs(pw[w, 3] - E.real) < RTOL * abs(E) and abs(pw[w, 4] - E.imag) < RTOL * abs(E)
        assert abs(pw[w, 5] - Nn.real) < RTOL * abs(Nn) and abs(pw[w, 6] - Nn.imag) < RTOL * abs(Nn)
    res = [afqmc.WalkerResult(st[-1].logw, st[-1].alive, st[-1].G, st[-1].logdet,
                              *afqmc.local_energy(s, st[-1].G)) for st in ref]
    E_ref, N_ref, _ = afqmc.weighted_estimate(res)
    assert abs(est["E"].real - E_ref) < RTOL * abs(E_ref)
    assert abs(est["N"].real - N_ref) < RTOL * abs(N_ref)
    assert p.status() == 0


@pytest.mark.parametrize("stab,order", [(0, 6), (1, 6), (5, 1), (3, 9)])
def test_parity_options(ftq, stab, order):
    """Stabilisation interval and Taylor order variants (N=2, M=7)."""
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 8
    f = gaussian_fields(99, s.n_slices, W, s.N_alpha)
    p = make(ftq, "ueg_n2_m7", W=W, stabilise_every=stab, exp_order=order)
    p.propagate(torch.from_numpy(f).cuda())
    G = p.green().cpu().numpy()
    ws = p.weights().cpu().numpy()
    o = afqmc.Options(stabilise_every=stab, exp_order=order)
    ref = oracle_states(s, f, o, s.n_slices, range(W))
    for w in range(W):
        assert_walker_close(G[w], ws[w], ref[w][-1], f"walker {w}")


def test_parity_free_projection(ftq):
    """Unconstrained weights: ln|w| and arg w (Eq. import, complex)."""
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 16
    f = gaussian_fields(7, s.n_slices, W, s.N_alpha)
    p = make(ftq, "ueg_n2_m7", W=W, constraint=ftq.FTQ_FREE)
    p.propagate(torch.from_numpy(f).cuda())
    ws = p.weights().cpu().numpy()
    ref = afqmc.run(s, f, afqmc.Options(constraint="free"))
    for w in range(W):
        lw = ref[w].logw
        assert abs(ws[w, 0] - lw.real) < RTOL * max(1, abs(lw.real))
        assert abs(math.remainder(ws[w, 1] - lw.imag, 2 * math.pi)) < 1e-9


def test_parity_config2_sampled(ftq):
    """N=14, M=57, whole path (87 slices) for 6 walkers, checked at slices
    10, 50 and 87 (ragged last tile of every 32-wide GEMM tile)."""
    c = WORKLOADS["ueg_n14_m57"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 6
    f = gaussian_fields(c["seed"], s.n_slices, W, s.N_alpha)
    p = make(ftq, "ueg_n14_m57", W=W)
    ref = oracle_states(s, f, afqmc.Options(), s.n_slices, range(W))
    fd = torch.from_numpy(f).cuda()
    done = 0
    for stop in (10, 50, s.n_slices):
        p.propagate(fd[done:stop].contiguous())
        done = stop
        G = p.green().cpu().numpy()
        ws = p.weights().cpu().numpy()
        for w in range(W):
            assert_walker_close(G[w], ws[w], ref[w][stop - 1], f"slice {stop} walker {w}")
    est = p.estimators()["per_walker"].cpu().numpy()
    for w in range(W):
        E, _ = afqmc.local_energy(s, ref[w][-1].G)
        assert abs(est[w, 3] - E.real) < RTOL * abs(E)


def test_full_size_sampled_walkers(ftq):
    """M=257, 1024 walkers (the benchmark's launch shape), 6 slices with one
    QRCP; walkers 0, 511 and 1023 against the oracle one by one."""
    c = WORKLOADS["ueg_n66_m257"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = c["walkers"]
    n = 6
    f = gaussian_fields(c["seed"], n, W, s.N_alpha)
    p = make(ftq, "ueg_n66_m257")
    p.propagate(torch.from_numpy(f).cuda())
    G = p.green()
    ws = p.weights().cpu().numpy()
    for w in (0, 511, 1023):
        ref = oracle_states(s, f, afqmc.Options(), n, [w])[0]
        assert_walker_close(G[w].cpu().numpy(), ws[w], ref[-1], f"walker {w}")
    assert p.status() == 0


def test_noninteracting_closed_form_full_size(ftq):
    """Zero fields keep G diagonal, so xbar = 0 and V = 0 exactly; the path
    is then free electrons with energies eps + delta_eps and
    G(beta) = diag(1 - f_FD), 2 ln det = ln Z_0.  M=257, beta=8.69, 348
    slices: every D_L / D_R scale of the headline workload."""
    c = WORKLOADS["ueg_n66_m257"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    W = 2
    p = make(ftq, "ueg_n66_m257", W=W)
    fz = torch.zeros((s.n_slices, W, s.N_alpha), dtype=torch.float64, device="cuda")
    p.propagate(fz)
    G = p.green().cpu().numpy()
    ws = p.weights().cpu().numpy()
    e = s.eps + s.delta_eps
    fd = fermi_dirac(e, s.mu, s.beta)
    ld = np.sum(np.log1p(np.exp(-s.beta * (e - s.mu))))
    for w in range(W):
        assert np.abs(G[w] - np.diag(1 - fd)).max() < 1e-11
        assert abs(ws[w, 3] - ld) < 1e-11 * ld
        assert ws[w, 2] > 0.5
    p.close()


def test_free_projection_vs_exact_diagonalisation(ftq):
    """GPU free projection with 8192 walkers reproduces ED <E>, <N>."""
    c = WORKLOADS["ueg_n2_m7"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    E_ed, N_ed = ed.grand_canonical(s)
    W = 8192
    f = gaussian_fields(2024, s.n_slices, W, s.N_alpha)
    p = make(ftq, "ueg_n2_m7", W=W, constraint=ftq.FTQ_FREE)
    p.propagate(torch.from_numpy(f).cuda())
    pw = p.estimators()["per_walker"].cpu().numpy()
    w = np.exp(pw[:, 0] - pw[:, 0].max() + 1j * pw[:, 1])
    E = pw[:, 3] + 1j * pw[:, 4]
    Nn = pw[:, 5] + 1j * pw[:, 6]
    blocks = np.array_split(np.arange(W), 32)
    Eb = np.array([(np.sum(w[b] * E[b]) / np.sum(w[b])).real for b in blocks])
    Nb = np.array([(np.sum(w[b] * Nn[b]) / np.sum(w[b])).real for b in blocks])
    Em, eE = (np.sum(w * E) / np.sum(w)).real, Eb.std() / math.sqrt(len(blocks))
    Nm, eN = (np.sum(w * Nn) / np.sum(w)).real, Nb.std() / math.sqrt(len(blocks))
    assert abs(Em - E_ed) < 3 * eE + 5e-3, (Em, eE, E_ed)
    assert abs(Nm - N_ed) < 3 * eN + 2e-3, (Nm, eN, N_ed)


def test_sequencing_errors(ftq):
    """Passing tau = beta is rejected; reset returns to tau = 0; an empty
    call is a no-op."""
    c = WORKLOADS["ueg_n2_m7"]
    p = make(ftq, "ueg_n2_m7", W=2)
    n = p.n_slices
    f = torch.zeros((n + 1, 2, p.n_alpha), dtype=torch.float64, device="cuda")
    with pytest.raises(ftq.FTQError):
        p.propagate(f)
    p.propagate(f[:0].contiguous())
    assert p.query("SLICE") == 0
    p.propagate(f[:n].contiguous())
    assert p.query("SLICE") == n
    p.reset()
    assert p.query("SLICE") == 0
    with pytest.raises(ftq.FTQError):
        p.propagate(torch.zeros((1, 3, p.n_alpha), dtype=torch.float64, device="cuda"))
