"""The library's on-device field generator (ftq_fields; used by
ftq_propagate_slices when no fields are passed) against the host
Philox4x32-10 / Box-Muller of synthetic_inputs, written independently from
the same published definition: the same counters give the same draws (up to
the last-bit differences of log / sincos), and a propagation with internal
fields equals one with the host draws passed in."""
import numpy as np
import pytest

from synthetic_inputs import WORKLOADS, philox_fields

torch = pytest.importorskip("torch")
stats = pytest.importorskip("scipy.stats")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ftq():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2012_12228_gb300 as m
    return m


def make(ftq, wl, W, seed, precision=None):
    c = WORKLOADS[wl]
    kw = {} if precision is None else dict(precision=precision)
    return ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, seed=seed, **kw)


@pytest.mark.parametrize("seed", [0, 7, (1 << 40) + 3])
def test_device_fields_match_host_generator(ftq, seed):
    p = make(ftq, "ueg_n14_m57", 48, seed)
    for first, n in ((0, 3), (40, 5), (p.n_slices - 2, 2)):
        x = p.fields(first, n).cpu().numpy()
        ref = philox_fields(seed, n, 48, p.n_alpha, first_slice=first)
        assert np.max(np.abs(x - ref)) < 1e-13 * max(1.0, np.max(np.abs(ref)))
    p.close()


def test_device_fields_are_standard_normal(ftq):
    p = make(ftq, "ueg_n66_m257", 256, 2026)
    x = p.fields(0, 20).cpu().numpy().ravel()
    p.close()
    n = x.size
    assert abs(x.mean()) < 5 / np.sqrt(n)
    assert abs(x.var() - 1) < 5 * np.sqrt(2 / n)
    assert stats.kstest(x[: 1 << 20], "norm").pvalue > 1e-3


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_internal_fields_propagation_equals_passed_fields(ftq, precision):
    prec = ftq.FTQ_FP64 if precision == "fp64" else ftq.FTQ_MIXED
    W, seed = 16, 4242
    a = make(ftq, "ueg_n14_m57", W, seed, prec)
    b = make(ftq, "ueg_n14_m57", W, seed, prec)
    n = 12
    a.propagate(n)
    b.propagate(torch.from_numpy(philox_fields(seed, n, W, b.n_alpha)).cuda())
    ga, gb = a.green().cpu().numpy(), b.green().cpu().numpy()
    wa, wb = a.weights().cpu().numpy(), b.weights().cpu().numpy()
    assert a.status() == 0 and b.status() == 0
    # the draws differ in the last bit at most (log / sincos); the FP32 chain
    # may round such a draw differently, hence the FP32-level bound there
    tol = 1e-9 if precision == "fp64" else 1e-5
    assert np.max(np.abs(ga - gb)) < tol * np.max(np.abs(gb))
    assert np.max(np.abs(wa[:, 0] - wb[:, 0])) < tol * max(1.0, np.max(np.abs(wb[:, 0])))
    assert np.array_equal(wa[:, 2], wb[:, 2])
    a.close()
    b.close()
