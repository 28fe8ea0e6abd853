"""Edge sizes on the GPU: one walker and an odd walker count (grids with a
single or ragged walker dimension) against the oracle and, for the mixed path,
against complex128; the largest basis of the mixed path (M = 1021, 7512
fields per slice) against the oracle on the complex128 path and the mixed
path against complex128 across a stabilisation (16-column Q panels, 8-column
QR panels); the paper's low-rank study basis M = 1189 (8852 fields) on the
complex128 path against the oracle; the limits (M = 1045 mixed, M = 2109
complex128) rejected."""
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


@pytest.mark.parametrize("W", [1, 3])
def test_single_and_odd_walker_counts(ftq, W):
    c = WORKLOADS["ueg_n14_m57"]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    n = 12
    f = gaussian_fields(c["seed"] + 70 + W, n, W, s.N_alpha)
    ref = afqmc.run(s, f, afqmc.Options(green="two_sided"), n_slices=n, want_estimator=False)
    fd = torch.from_numpy(f).cuda()
    out = {}
    for prec in (ftq.FTQ_FP64, ftq.FTQ_MIXED):
        p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, precision=prec)
        p.propagate(fd)
        out[prec] = (p.green().cpu().numpy(), p.weights().cpu().numpy())
        assert p.status() == 0
        p.close()
    G, ws = out[ftq.FTQ_FP64]
    for w in range(W):
        assert np.abs(G[w] - ref[w].G).max() < 1e-10 * np.abs(ref[w].G).max()
        assert abs(ws[w, 0] - ref[w].logw.real) < 1e-9 * max(1.0, abs(ref[w].logw.real))
    Gm, wm = out[ftq.FTQ_MIXED]
    assert np.abs(Gm - G).max() < 1e-5 * np.abs(G).max()


@pytest.mark.timeout(900)
def test_largest_basis_complex128(ftq):
    N, M, rs, theta, dtau = 14, 1021, 0.5, 0.125, 0.05
    s = UEG(N, M, rs, theta, dtau)
    n, W = 6, 2
    f = gaussian_fields(1250, n, W, s.N_alpha)
    p = ftq.Propagator(N, M, rs, theta, dtau, walkers=W, precision=ftq.FTQ_FP64)
    assert p.M == M and p.n_alpha == s.N_alpha
    p.propagate(torch.from_numpy(f).cuda())
    G = p.green().cpu().numpy()
    ws = p.weights().cpu().numpy()
    assert p.status() == 0
    p.close()
    ref = afqmc.run(s, f, afqmc.Options(green="two_sided"), n_slices=n, want_estimator=False)
    for w in range(W):
        assert np.abs(G[w] - ref[w].G).max() < 1e-10 * np.abs(ref[w].G).max()
        assert abs(ws[w, 0] - ref[w].logw.real) < 1e-9 * max(1.0, abs(ref[w].logw.real))
    with pytest.raises(ftq.FTQError):
        ftq.Propagator(N, 1045, rs, theta, dtau, walkers=1, precision=ftq.FTQ_MIXED)


@pytest.mark.timeout(900)
def test_largest_basis_mixed(ftq):
    """M = 1021, 2 walkers, 6 slices (one stabilisation): mixed vs complex128."""
    N, M, rs, theta, dtau = 14, 1021, 0.5, 0.125, 0.05
    s = UEG(N, M, rs, theta, dtau)
    n, W = 6, 2
    f = torch.from_numpy(gaussian_fields(1251, n, W, s.N_alpha)).cuda()
    out = {}
    for prec in (ftq.FTQ_FP64, ftq.FTQ_MIXED):
        p = ftq.Propagator(N, M, rs, theta, dtau, walkers=W, precision=prec)
        p.propagate(f)
        out[prec] = (p.green().cpu().numpy(), p.weights().cpu().numpy())
        assert p.status() == 0
        p.close()
    (Ga, wa), (Gb, wb) = out[ftq.FTQ_FP64], out[ftq.FTQ_MIXED]
    err = np.abs(Ga - Gb).max() / np.abs(Ga).max()
    print(f"M=1021 mixed vs complex128 after 6 slices: G rel {err:.2e}")
    assert err < 1e-5
    # ln det sums the logs of M FP32 LU pivots, each a few ulps (2^-23) off:
    # an absolute error of at most M 2^-20 (|ln det| is only ~25 here, most of
    # the 1021 orbitals being nearly empty)
    dld = np.abs(wa[:, 3] - wb[:, 3]).max()
    print(f"M=1021 ln det abs diff {dld:.2e} (bound {M * 2.0 ** -20:.2e})")
    assert dld < M * 2.0 ** -20


@pytest.mark.timeout(1200)
def test_basis_1189_complex128(ftq):
    """N=14, M=1189, r_s=0.5, Theta=0.125 (the basis of the paper's low-rank
    compression study): one walker, one slice, against the oracle."""
    N, M, rs, theta, dtau = 14, 1189, 0.5, 0.125, 0.01
    s = UEG(N, M, rs, theta, dtau)
    f = gaussian_fields(1252, 1, 1, s.N_alpha)
    p = ftq.Propagator(N, M, rs, theta, dtau, walkers=1, precision=ftq.FTQ_FP64)
    assert p.M == M and p.n_alpha == s.N_alpha == 8852
    p.propagate(torch.from_numpy(f).cuda())
    G = p.green().cpu().numpy()[0]
    ws = p.weights().cpu().numpy()[0]
    assert p.status() == 0
    p.close()
    ref = afqmc.run(s, f, afqmc.Options(green="two_sided"), n_slices=1, want_estimator=False)[0]
    assert np.abs(G - ref.G).max() < 1e-10 * np.abs(ref.G).max()
    assert abs(ws[3] - ref.logdet.real) < 1e-10 * abs(ref.logdet.real)
    with pytest.raises(ftq.FTQError):
        ftq.Propagator(N, 2109, rs, theta, dtau, walkers=1, precision=ftq.FTQ_FP64)
