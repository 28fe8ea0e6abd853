"""Edge sizes on the GPU: one walker and an odd walker count (grids with a
single or ragged walker dimension) against the oracle and, for the mixed path,
against complex128; the largest basis the library accepts (M = 1021, the last
closed shell below its limit of 1024, 7512 fields per slice) against the
oracle on the complex128 path; M = 1045 is rejected."""
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
        ftq.Propagator(N, 1045, rs, theta, dtau, walkers=1)
