"""Ragged batch (several UEG systems of different basis size in one
persistent tensor-core launch per Horner step, CUDA-graph-captured) against
independent single-system contexts on identical fields, and the autotuner.

The batched kernel performs, for every work item, exactly the arithmetic of
the single-system launch (same operands, same k order, same epilogue), so G,
the weights and the log-determinants must agree to rounding (1e-6 relative,
the mixed path's own tolerance, is asserted)."""
import numpy as np
import pytest

from synthetic_inputs import RAGGED, gaussian_fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ftq():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2012_12228_gb300 as m
    return m


def small_systems():
    out = []
    for sd, W in zip(RAGGED, (8, 4, 3, 2)):
        d = dict(sd)
        d["walkers"] = W
        out.append(d)
    return out


def fields_for(systems, n, first=0):
    from oracle.ueg import UEG
    fl = []
    for sd in systems:
        na = UEG(sd["N"], sd["M"], sd["rs"], sd["theta"], sd["dtau"]).N_alpha
        fl.append(torch.from_numpy(gaussian_fields(sd["seed"], n, sd["walkers"], na, first_slice=first)).cuda())
    return fl


def test_batch_matches_single_contexts(ftq):
    systems = small_systems()
    n = 7                                    # crosses the QRCP at slice 5
    fl = fields_for(systems, n)
    b = ftq.Batch(systems)
    b.propagate([f[:3].contiguous() for f in fl])        # two calls: the graph is updated and replayed
    b.propagate([f[3:].contiguous() for f in fl])
    for sd, f, m in zip(systems, fl, b.members):
        p = ftq.Propagator(sd["N"], sd["M"], sd["rs"], sd["theta"], sd["dtau"], walkers=sd["walkers"],
                           precision=ftq.FTQ_MIXED)
        p.propagate(f)
        Ga, Gb = p.green().cpu().numpy(), m.green().cpu().numpy()
        wa, wb = p.weights().cpu().numpy(), m.weights().cpu().numpy()
        err = np.abs(Ga - Gb).max() / np.abs(Ga).max()
        print(f"M={sd['M']}: batch vs single G rel err {err:.2e}")
        assert err < 1e-6
        assert np.allclose(wa[:, [0, 2, 3]], wb[:, [0, 2, 3]], rtol=1e-6, atol=1e-6)
        assert m.status() == 0
        p.close()
    b.close()


def test_autotune_keeps_results(ftq):
    systems = small_systems()
    fl = fields_for(systems, 6)
    a = ftq.Batch(systems)
    a.propagate(fl)
    b = ftq.Batch(systems)
    choice = b.autotune()
    print("autotuned column tiles (tiles, ms per Horner step):", choice)
    assert all(c[0] in (1, 2, 3) and c[1] > 0 for c in choice)
    b.propagate(fl)
    for ma, mb in zip(a.members, b.members):
        Ga, Gb = ma.green().cpu().numpy(), mb.green().cpu().numpy()
        assert np.abs(Ga - Gb).max() / np.abs(Ga).max() < 1e-5
    a.close()
    b.close()


def test_batch_rejects_passing_beta(ftq):
    systems = small_systems()
    b = ftq.Batch(systems)
    n0 = min(m.n_slices for m in b.members)
    fl = fields_for(systems, n0 + 1)
    with pytest.raises(ftq.FTQError):
        b.propagate(fl)
    b.close()
