"""The update of T^-1 at each stabilisation of the mixed path runs in
double-FP32 arithmetic on the FP32 pipe (FTQ_MIXED).  FTQ_MIXED_F64UDT runs
the same update on the FP64 pipe; everything else is the same code.

N=2, M=7, 16 walkers, the whole 22-slice path (four stabilisations): the FP32
slice quantities round identically in the two modes (the two T^-1 differ by
about 1e-14 relative, far below the FP32 rounding of the per-slice Green's
function), so G(beta), ln det and ln|w| at tau = beta, which use T^-1 in
complex128, agree to 1e-12.  At N=66, M=257 (1024 walkers, two
stabilisations) the paths agree to the FP32 accuracy of the slices."""
import numpy as np
import pytest

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


def run(ftq, wl, W, n, prec):
    c = WORKLOADS[wl]
    s = UEG(c["N"], c["M"], c["rs"], c["theta"], c["dtau"])
    f = torch.from_numpy(gaussian_fields(c["seed"], n, W, s.N_alpha)).cuda()
    p = ftq.Propagator(c["N"], c["M"], c["rs"], c["theta"], c["dtau"], walkers=W, precision=prec)
    p.propagate(f)
    out = (p.green()[::97].cpu().numpy(), p.weights().cpu().numpy())      # walkers 0, 97, ...
    assert p.status() == 0
    p.close()
    return out


def test_double_float_udt_equals_fp64_udt_config1(ftq):
    (Ga, wa), (Gb, wb) = (run(ftq, "ueg_n2_m7", 16, 22, prec) for prec in (ftq.FTQ_MIXED, ftq.FTQ_MIXED_F64UDT))
    eg = np.abs(Ga - Gb).max() / np.abs(Gb).max()
    ed = np.abs(wa[:, 3] - wb[:, 3]).max() / np.abs(wb[:, 3]).max()
    print(f"M=7 double-FP32 vs FP64 T^-1 update: G(beta) {eg:.1e}, ln det {ed:.1e}")
    assert np.array_equal(wa[:, 2], wb[:, 2])
    assert eg < 1e-12 and ed < 1e-12
    assert np.abs(wa[:, 0] - wb[:, 0]).max() < 1e-12 * max(1.0, np.abs(wb[:, 3]).max())


def test_double_float_udt_full_size(ftq):
    (Ga, wa), (Gb, wb) = (run(ftq, "ueg_n66_m257", 1024, 10, prec)
                          for prec in (ftq.FTQ_MIXED, ftq.FTQ_MIXED_F64UDT))
    eg = max(np.abs(a - b).max() / np.abs(b).max() for a, b in zip(Ga, Gb))
    ed = np.abs(wa[:, 3] - wb[:, 3]).max() / np.abs(wb[:, 3]).max()
    print(f"M=257 double-FP32 vs FP64 T^-1 update, 10 slices: G {eg:.1e}, ln det {ed:.1e}")
    assert eg < 1e-5 and ed < 1e-5
