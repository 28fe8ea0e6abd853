"""Failure detection with faults made on the host (no GPU fault): a NaN in one
walker's auxiliary fields latches FTQ_ENUMERIC (-3) in the device status
word and drops that walker (weight 0), the other walkers' results equal
those of a clean run, the estimators stay finite, the comb's parents equal
the oracle comb's on the same weights, reading the status clears it, and
after a reset the context runs the clean fields to the same results again
(complex128 and mixed precision)."""
import numpy as np
import pytest

from oracle.population import comb_counts, comb_pairs
from synthetic_inputs import WORKLOADS, gaussian_fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FTQ_ENUMERIC = -3
FTQ_ETIMEOUT = -4


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
    assert w1[bad, 2] == 0.0                                 # the walker is dropped
    for w in range(W):
        if w != bad:
            assert np.array_equal(G1[w], G0[w])
            assert np.array_equal(w1[w, :3], w0[w, :3])
    est = p.estimators()
    assert np.isfinite(est["E"].real) and np.isfinite(est["N"].real)
    assert est["n_alive"] == int(np.sum(w1[:, 2] > 0.5))
    # comb on the same weights as the oracle comb (non-finite or dead: weight 0)
    xi = 0.37
    ok = (w1[:, 2] > 0.5) & np.isfinite(w1[:, 0])
    lw = np.where(ok, w1[:, 0], -np.inf)
    wts = np.where(ok, np.exp(lw - lw.max()), 0.0)
    C = np.cumsum(wts)
    teeth = (np.arange(W) + xi) * (C[-1] / W)
    assert np.min(np.abs(teeth[:, None] - C[None, :])) > 1e-9
    parent_ref = list(range(W))
    for src, dst in comb_pairs(comb_counts(wts, xi)):
        parent_ref[dst] = src
    parent = p.population_control(xi).cpu().numpy()
    assert list(parent) == parent_ref
    assert p.status() == 0
    p.reset()
    p.propagate(clean)
    assert np.array_equal(p.green().cpu().numpy(), G0)
    assert p.status() == 0
    p.close()


@pytest.mark.parametrize("green_kernel", [2, 1])
def test_chain_wait_that_runs_out_latches_timeout(ftq, green_kernel):
    """The tensor-core kernels' bounded mbarrier waits, cut to zero polls by
    the test hook, give up at once: the launch latches FTQ_ETIMEOUT, skips its
    work, drains its own copies and MMAs with the normal bound and frees its
    tensor memory; after a reset the same context reproduces a clean run
    exactly.  With green_kernel = 1 the slice's G(tau) also comes from the
    tensor-core Gauss-Jordan kernel, whose MMA wait gives up the same way.
    (N=2, M=7, 4 walkers: the smallest launch.)"""
    c = WORKLOADS["ueg_n2_m7"]
    W, n = 4, 6
    ref = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, precision=ftq.FTQ_MIXED)
    ref.set_green_kernel(green_kernel)
    f = torch.from_numpy(gaussian_fields(c["seed"], n, W, ref.n_alpha)).cuda()
    ref.propagate(f)
    G0, w0 = ref.green().cpu().numpy(), ref.weights().cpu().numpy()
    assert ref.status() == 0
    ref.close()
    p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, precision=ftq.FTQ_MIXED)
    p.set_green_kernel(green_kernel)
    p.set_wait_limit(0)
    p.propagate(f[:1].contiguous())
    torch.cuda.synchronize()
    assert p.status() == FTQ_ETIMEOUT
    assert p.status() == 0
    p.set_wait_limit(-1)
    p.reset()
    p.propagate(f)
    assert np.array_equal(p.green().cpu().numpy(), G0)
    assert np.array_equal(p.weights().cpu().numpy(), w0)
    assert p.status() == 0
    with pytest.raises(ftq.FTQError):
        p.set_wait_limit(-2)
    p.close()
