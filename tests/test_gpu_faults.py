"""Failure detection with faults made on the host (no GPU fault): a NaN in one
walker's auxiliary fields latches FTQ_ENUMERIC (-3) in the device status
word, the other walkers' results equal those of a clean run, reading the
status clears it, and after a reset the context runs the clean fields to
the same results again (complex128 and mixed precision)."""
import numpy as np
import pytest

from synthetic_inputs import WORKLOADS, gaussian_fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FTQ_ENUMERIC = -3


@pytest.fixture(scope="module")
def ftq():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2012_12228_gb300 as m
    return m


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_nan_field_latches_numeric_status(ftq, prec):
    c = WORKLOADS["ueg_n14_m57"]
    W, n, bad = 4, 10, 1
    p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W,
                       precision=ftq.FTQ_FP64 if prec == "fp64" else ftq.FTQ_MIXED)
    f = gaussian_fields(c["seed"] + 80, n, W, p.n_alpha)
    clean = torch.from_numpy(f).cuda()
    p.propagate(clean)
    G0, w0 = p.green().cpu().numpy(), p.weights().cpu().numpy()
    assert p.status() == 0
    p.reset()
    f_bad = f.copy()
    f_bad[3, bad, 5] = np.nan
    p.propagate(torch.from_numpy(f_bad).cuda())
    G1, w1 = p.green().cpu().numpy(), p.weights().cpu().numpy()
    assert p.status() == FTQ_ENUMERIC
    assert p.status() == 0                                   # reading cleared the latch
    assert not np.all(np.isfinite(G1[bad]))
    for w in range(W):
        if w != bad:
            assert np.array_equal(G1[w], G0[w])
            assert np.array_equal(w1[w, :3], w0[w, :3])
    p.reset()
    p.propagate(clean)
    assert np.array_equal(p.green().cpu().numpy(), G0)
    assert p.status() == 0
    p.close()
