"""The two G(tau_k) kernels of the mixed path, the tensor-core Gauss-Jordan
kernel (rank-16 updates as tcgen05 3xTF32 MMAs) and the CUDA-core blocked LU,
against the oracle and against each other on interacting fields.

* each kernel forced on M = 7, 57, 123 and 257 (one 64-row MMA tile with a
  ragged tail, one, two, and four plus a single row; the last 16-column
  panel ragged in every case), four walkers over 12 slices (two
  stabilisations): G(tau_12), ln det(I + A_12) and ln|w| of walkers 0 and 3
  against the oracle;
* the two kernels against each other on the same fields;
* M = 515, where the tensor-core kernel is the default: two walkers over
  12 slices against the oracle;
* ftq_autotune picks one of the two and leaves G, the weights and the status
  word as they were.

Tolerances as in the other mixed-path tests: the chain holds hi + lo tf32
planes (relative 2^-22 per rounding) and both G kernels eliminate in FP32,
so G is held to 1e-4 relative.  ln det(I + A_k) is a sum of M FP32
log-pivots on top of the chain's rounding, so its absolute error grows like
M 2^-20 whatever its size: it is held to the larger of 1e-5 |ln det| (paths
of up to 12 slices) and M 2^-20, and ln|w| (whose real part telescopes to
twice ln det) to twice that.  Against each other the kernels differ only by the
FP32 rounding of two pivoted eliminations of the same well-conditioned
matrix (the chain is identical), so G agrees to 1e-5 relative and ln det to
1e-6 relative.
"""
import numpy as np
import pytest

from oracle.ueg import UEG
from oracle_pool import Checkpoints
from synthetic_inputs import WORKLOADS, gaussian_fields

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TC, LU = 1, 2
M515 = dict(N=14, M=515, rs=0.5, theta=0.125, dtau=0.05, seed=1401)


@pytest.fixture(scope="module")
def ftq():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2012_12228_gb300 as m
    return m


def _sys(c):
    return UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])


def _run(ftq, c, f, kind):
    p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=f.shape[1],
                       precision=ftq.FTQ_MIXED)
    p.set_green_kernel(kind)
    assert p.query("GREEN_KERNEL") == kind
    p.propagate(torch.from_numpy(f).cuda())
    out = (p.green().cpu().numpy(), p.weights().cpu().numpy())
    assert p.status() == 0
    p.close()
    return out


def _check(label, G, ws, w, ref_trace, n, M):
    k, Gr, lw, alive, ld = ref_trace[-1]
    assert k == n
    eg = np.abs(G[w] - Gr).max() / np.abs(Gr).max()
    ed = abs(ws[w, 3] - ld.real)
    el = abs(ws[w, 0] - lw.real) if alive else 0.0
    tol = max(1e-5 * max(1.0, abs(ld.real)), M * 2.0 ** -20)
    print(f"{label} walker {w}: G rel {eg:.2e}, ln det abs {ed:.2e} (|ln det| {abs(ld.real):.1f}, "
          f"bound {tol:.1e}), ln|w| abs {el:.2e}")
    assert bool(ws[w, 2] > 0.5) == bool(alive)
    assert eg < 1e-4
    assert ed < tol
    assert el < 2 * tol


@pytest.mark.parametrize("wl", ["ueg_n2_m7", "ueg_n14_m57", "ueg_n14_m123", "ueg_n66_m257"])
def test_both_green_kernels_vs_oracle(ftq, wl):
    c = WORKLOADS[wl]
    s = _sys(c)
    n, W = 12, 4
    f = gaussian_fields(c["seed"] + 77, n, W, s.N_alpha)
    oracle = Checkpoints([(c, f[:, 0, :]), (c, f[:, W - 1, :])], [n], n)
    out = {kind: _run(ftq, c, f, kind) for kind in (TC, LU)}
    ref = oracle.get()
    for kind, (G, ws) in out.items():
        for i, (trace, _) in enumerate(ref):
            _check(f"M={c['M']} {'tensor-core GJ' if kind == TC else 'CUDA-core LU'}", G, ws, (0, W - 1)[i],
                   trace, n, c["M"])
    (Ga, wa), (Gb, wb) = out[TC], out[LU]
    eg = np.abs(Ga - Gb).max() / np.abs(Gb).max()
    ed = (np.abs(wa[:, 3] - wb[:, 3]) / np.maximum(1.0, np.abs(wb[:, 3]))).max()
    print(f"M={c['M']}: tensor-core GJ vs CUDA-core LU, G rel {eg:.2e}, ln det rel {ed:.2e}")
    assert eg < 1e-5
    assert ed < 1e-6


def test_tensor_core_green_m515_vs_oracle(ftq):
    c = M515
    s = _sys(c)
    n, W = 12, 2
    f = gaussian_fields(c["seed"], n, W, s.N_alpha)
    oracle = Checkpoints([(c, f[:, w, :]) for w in range(W)], [n], n)
    p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, precision=ftq.FTQ_MIXED)
    assert p.query("GREEN_KERNEL") == TC                 # the default from M = 384 up
    p.propagate(torch.from_numpy(f).cuda())
    G, ws = p.green().cpu().numpy(), p.weights().cpu().numpy()
    assert p.status() == 0
    p.close()
    for w, (trace, _) in enumerate(oracle.get()):
        _check("M=515 tensor-core GJ", G, ws, w, trace, n, c["M"])


def test_autotune_chooses_a_green_kernel_without_side_effects(ftq):
    c = WORKLOADS["ueg_n14_m57"]
    s = _sys(c)
    W = 64
    f = torch.from_numpy(gaussian_fields(c["seed"], 3, W, s.N_alpha)).cuda()
    p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, precision=ftq.FTQ_MIXED)
    p.propagate(f)
    G0, w0 = p.green().cpu().numpy(), p.weights().cpu().numpy()
    p.autotune()
    assert p.query("GREEN_KERNEL") in (TC, LU)
    G1, w1 = p.green().cpu().numpy(), p.weights().cpu().numpy()
    assert np.array_equal(G0, G1)
    assert np.array_equal(w0, w1)
    assert p.status() == 0
    p.close()
