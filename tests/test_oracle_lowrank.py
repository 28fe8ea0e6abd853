"""Pins of the low-rank truncation (Sec. "Exploiting the low-rank structure",
Eq. thresh, reading T) in the oracle against what the definition and the
mathematics fix:

* nothing truncated (threshold below every scale): the Woodbury G and the
  determinant lemma equal the full-rank stable G and ln det along whole paths;
* truncated: G and ln det equal (I + R_tr D_L,tr)^-1 and ln det(I + R_tr
  D_L,tr) formed directly, with R_tr the kept right factors and D_L,tr the
  left block with its entries below the threshold set to zero;
* the right-block truncation keeps exactly the leading |R_jj| >= threshold of
  the pivoted QR, and the rank never grows;
* at the paper's threshold 1e-6 the energy and number differ from full rank by
  far less than the statistical resolution, while the rank drops at low
  temperature.
"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import afqmc
from oracle.ueg import UEG
from synthetic_inputs import gaussian_fields


def clogdet(A):
    sign, la = np.linalg.slogdet(A)
    return la + 1j * np.angle(sign)


def wrap(a):
    return math.remainder(a, 2 * math.pi)


def cfg2():
    return UEG(14, 57, 1.0, 0.125, 0.05)


@pytest.mark.parametrize("which,n", [("cfg1", None), ("cfg2", 12)])
def test_untruncated_equals_full_rank(which, n):
    s = UEG(2, 7, 1.0, 0.5, 0.05) if which == "cfg1" else cfg2()
    f = gaussian_fields(51, s.n_slices, 2, s.N_alpha)
    full = afqmc.run(s, f, afqmc.Options(green="two_sided"), n_slices=n)
    lr = afqmc.run(s, f, afqmc.Options(low_rank=1e-300), n_slices=n)
    for a, b in zip(full, lr):
        assert np.abs(a.G - b.G).max() < 1e-10 * np.abs(a.G).max()
        assert abs(a.logdet.real - b.logdet.real) < 1e-10 * max(1.0, abs(a.logdet.real))
        assert abs(wrap(a.logdet.imag - b.logdet.imag)) < 1e-10
        assert abs(a.logw.real - b.logw.real) < 1e-9 * max(1.0, abs(a.logw.real))


def _state_at(s, f, k, thr):
    o = afqmc.Options(low_rank=thr)
    st = afqmc.initial_state(s)
    for j in range(1, k + 1):
        st, *_ = afqmc.slice_step(s, st, f[j - 1], j, o)
    return st


@pytest.mark.parametrize("k,thr", [(20, 1e-3), (75, 1e-3), (80, 1e-6)])
def test_truncated_green_equals_definition(k, thr):
    s = cfg2()
    f = gaussian_fields(52, s.n_slices, 1, s.N_alpha)[:, 0]
    st = _state_at(s, f, k, thr)
    DL = afqmc.left_diagonal(s, k)
    DLt = np.where(DL >= thr, DL, 0.0)
    A = (st.Y * st.D[None, :]) @ st.T * DLt[None, :]
    I = np.eye(s.M)
    m_left = int(np.sum(DL >= thr))
    assert len(st.D) < s.M or m_left < s.M          # something is truncated
    G, ld = afqmc.green_lowrank(DL, st.Y, st.D, st.T, thr)
    assert np.abs(G - np.linalg.inv(I + A)).max() < 1e-9 * np.abs(G).max()
    ref = clogdet(I + A)
    assert abs(ld.real - ref.real) < 1e-9 * max(1.0, abs(ref.real))
    assert abs(wrap(ld.imag - ref.imag)) < 1e-9
    assert np.abs(st.G - G).max() == 0.0              # the path used the same G


def test_right_truncation_keeps_the_leading_scales():
    s = cfg2()
    f = gaussian_fields(53, s.n_slices, 1, s.N_alpha)[:, 0]
    thr = 1e-3
    o = afqmc.Options(low_rank=thr)
    st = afqmc.initial_state(s)
    ranks = []
    for j in range(1, s.n_slices + 1):
        if j % 5 == 0:
            C = st.Y * st.D[None, :]
            B = afqmc.propagator(s, f[j - 1] - afqmc.force_bias(s, st.G), o.exp_order)
            _, R, _ = sla.qr(B @ C, pivoting=True, mode="economic")
            d = np.abs(np.diag(R))
        st, *_ = afqmc.slice_step(s, st, f[j - 1], j, o)
        ranks.append(len(st.D))
        if j % 5 == 0:
            m = len(st.D)
            assert np.all(np.abs(st.D) >= thr)
            assert np.allclose(np.abs(st.D), d[:m], rtol=1e-10)
            if m < len(d):
                assert d[m] < thr
            assert st.Y.shape == (s.M, m) and st.T.shape == (m, s.M)
    assert all(a >= b for a, b in zip(ranks, ranks[1:]))
    assert ranks[-1] < s.M


def test_untruncated_stabilisation_equals_full():
    s = cfg2()
    f = gaussian_fields(54, 5, 1, s.N_alpha)[:, 0]
    st = _state_at(s, f, 4, 1e-300)
    B = afqmc.propagator(s, f[4] - afqmc.force_bias(s, st.G), 6)
    Y = B @ st.Y
    a = afqmc.stabilise(Y, st.D, st.T)
    b = afqmc.stabilise_truncated(Y, st.D, st.T, 1e-300)
    for x, y in zip(a, b):
        assert np.abs(x - y).max() < 1e-12 * np.abs(x).max()


def test_paper_threshold_accuracy_and_compression():
    s = cfg2()
    f = gaussian_fields(55, s.n_slices, 2, s.N_alpha)
    full = afqmc.run(s, f, afqmc.Options())
    lr = afqmc.run(s, f, afqmc.Options(low_rank=1e-6), record=True)
    for a, b in zip(full, lr):
        assert a.alive and b.alive
        assert abs(a.energy - b.energy) < 1e-5 * abs(a.energy)
        assert abs(a.number - b.number) < 1e-5 * abs(a.number)
        assert np.abs(a.G - b.G).max() < 1e-5
        assert b.rank_trace[0] == s.M and b.rank_trace[-1] < 0.7 * s.M


def test_untruncated_modified_overlap_equals_full_rank():
    """The low-rank Green's function also serves the modified overlap (trial
    block B_T^n at every slice, physical G(beta) and the final ratio): with a
    threshold below every scale it reproduces the full-rank modified path."""
    s = UEG(2, 7, 1.0, 0.5, 0.05)
    f = gaussian_fields(56, s.n_slices, 3, s.N_alpha)
    for constraint in ("phaseless", "free"):
        a = afqmc.run(s, f, afqmc.Options(overlap="modified", constraint=constraint, green="two_sided"))
        b = afqmc.run(s, f, afqmc.Options(overlap="modified", constraint=constraint, low_rank=1e-300))
        for x, y in zip(a, b):
            assert np.abs(x.G - y.G).max() < 1e-10 * np.abs(x.G).max()
            assert abs(x.logw.real - y.logw.real) < 1e-9 * max(1.0, abs(x.logw.real))
            assert abs(wrap(x.logw.imag - y.logw.imag)) < 1e-9
