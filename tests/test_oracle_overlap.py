"""Pins of the modified overlap ratio (Eq. ztfix, reading S) in the oracle
against what its definition fixes, with every product and determinant formed
directly (no stabilisation, no stable-G algebra):

* S~_k = [det(I + B_T^n R_k) / det(I + B_T^n R_{k-1})]^2 at every slice, the
  force bias from (I + R_{k-1} B_T^n)^-1, the phaseless weight of those ratios
  and the final ratio r, and G(beta) = (I + R_n)^-1;
* free projection with no force bias: the weight and G(beta) equal those of
  Eq. ftoratio (both telescope to the same determinants);
* the optimal force bias of S~ cancels the O(sqrt(dtau)) term of ln I_k.
"""
import math

import numpy as np
import pytest

from oracle import afqmc
from oracle.ueg import UEG
from synthetic_inputs import gaussian_fields


def cfg1():
    return UEG(2, 7, 1.0, 0.5, 0.05)


def clogdet(A):
    sign, la = np.linalg.slogdet(A)
    return la + 1j * np.angle(sign)


def wrap(a):
    return math.remainder(a, 2 * math.pi)


@pytest.mark.parametrize("seed", [31, 32])
def test_modified_ratios_match_direct_determinants(seed):
    s = cfg1()
    o = afqmc.Options(overlap="modified")
    f = gaussian_fields(seed, s.n_slices, 1, s.N_alpha)[:, 0]
    r = afqmc.propagate_walker(s, f, o, record=True, want_estimator=False)
    DL = afqmc.left_diagonal(s, 0)                     # B_T^n at every slice
    I = np.eye(s.M)
    R = np.eye(s.M, dtype=np.complex128)
    ld_prev = clogdet(I + DL[:, None] * R)
    logw, alive = 0.0, True
    for k in range(s.n_slices):
        Gt = np.linalg.inv(I + R * DL[None, :])        # (I + R_{k-1} B_T^n)^-1
        xb = afqmc.force_bias(s, Gt)
        assert np.abs(r.xbar_trace[k] - xb).max() < 1e-11 * max(1.0, np.abs(xb).max())
        R = afqmc.propagator(s, f[k] - xb, o.exp_order) @ R
        ld = clogdet(I + DL[:, None] * R)
        lnS = 2.0 * (ld - ld_prev)
        ld_prev = ld
        assert abs(r.lnS_trace[k].real - lnS.real) < 1e-10 * max(1.0, abs(lnS.real))
        assert abs(wrap(r.lnS_trace[k].imag - lnS.imag)) < 1e-10
        gauss = np.sum(f[k] * xb - 0.5 * xb * xb)
        if alive:
            c = math.cos(lnS.imag)
            if c <= 0.0:
                alive = False
            else:
                logw += lnS.real + gauss.real + math.log(c)
    lnr = 2.0 * (clogdet(I + R) - ld_prev)             # det(I + R_n) / det(I + B_T^n R_n)
    if alive:
        c = math.cos(lnr.imag)
        alive = c > 0.0
        logw += lnr.real + math.log(c) if alive else 0.0
    assert r.alive == alive
    if alive:
        assert abs(r.logw.real - logw) < 1e-10 * max(1.0, abs(logw))
    assert np.abs(r.G - np.linalg.inv(I + R)).max() < 1e-11
    ldr = clogdet(I + R)
    assert abs(r.logdet.real - ldr.real) < 1e-10 * max(1.0, abs(ldr.real))
    assert abs(wrap(r.logdet.imag - ldr.imag)) < 1e-10


def test_free_projection_without_bias_equals_paper_overlap():
    s = cfg1()
    f = gaussian_fields(33, s.n_slices, 4, s.N_alpha)
    out = {}
    for ov in ("paper", "modified"):
        out[ov] = afqmc.run(s, f, afqmc.Options(constraint="free", force_bias=False, overlap=ov))
    for a, b in zip(out["paper"], out["modified"]):
        assert abs(a.logw.real - b.logw.real) < 1e-10 * max(1.0, abs(a.logw.real))
        assert abs(wrap(a.logw.imag - b.logw.imag)) < 1e-10
        assert np.abs(a.G - b.G).max() < 1e-12
        assert abs(a.energy - b.energy) < 1e-10 * abs(a.energy)
    # with the phaseless constraint the two overlaps weigh the same path differently
    ph = [afqmc.run(s, f, afqmc.Options(force_bias=False, overlap=ov)) for ov in ("paper", "modified")]
    assert max(abs(a.logw.real - b.logw.real) for a, b in zip(*ph) if a.alive and b.alive) > 1e-6


@pytest.mark.parametrize("seed,kk", [(5, 6), (6, 12), (8, 18)])
def test_modified_force_bias_cancels_linear_term(seed, kk):
    """Reading P applied to S~: d ln I_k / dx at x = 0 is O(dtau), far below
    |xbar| = O(sqrt(dtau)), where with no shift it is about |xbar|.  (That the
    shift is the one of (I + R B_T^n)^-1 is pinned directly above.)"""
    s = cfg1()
    f = gaussian_fields(seed, s.n_slices, 1, s.N_alpha)[:, 0]
    o = afqmc.Options(overlap="modified", green="two_sided")
    st = afqmc.initial_state(s)
    for k in range(1, kk):
        st, *_ = afqmc.slice_step(s, st, f[k - 1], k, o)

    def grad(xbar):
        def lnI(x):
            _, lnS, _, _ = afqmc.slice_step(s, st, x, kk, o, xbar=xbar)
            return lnS + np.sum(x * xbar - 0.5 * xbar * xbar)
        h = 1e-5
        return np.array([(lnI(h * e) - lnI(-h * e)) / (2 * h) for e in np.eye(s.N_alpha)])

    xbar = afqmc.force_bias(s, st.G)
    nb = np.linalg.norm(xbar)
    assert nb > 1e-2
    assert np.linalg.norm(grad(xbar)) < 0.3 * nb
    assert np.linalg.norm(grad(0.0 * xbar)) > 0.8 * nb
