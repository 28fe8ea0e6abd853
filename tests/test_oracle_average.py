"""Pins of the oracle's time-slice estimates and their average (Results,
"Assessing the Phaseless Constraint": the global estimate at tau = beta,
"No Average", against the global estimate averaged over the time slices,
"Average").

The estimate after slice k uses the walkers' weights at slice k and the
local values from G(tau_k) = (I + R_k B_T^(n-k))^-1 (reading P).  Without a
constraint the propagators average to e^{-k dtau (H - mu N)}, so the
estimate at slice k approaches the exact mixed ratio
tr(e^{-k dtau (H - mu N)} e^{-(n-k) dtau H_T} O) / tr(...), computed here by
exact diagonalisation in Fock space (oracle.ed.mixed_estimate).
"""
import math

import numpy as np
import pytest

from oracle import afqmc, ed
from oracle.ueg import UEG, fermi_dirac
from synthetic_inputs import gaussian_fields


def cfg1():
    return UEG(2, 7, 1.0, 0.5, 0.05)


def test_mixed_estimate_end_points():
    """a = beta, b = 0 is the grand-canonical ensemble; a = 0, b = beta is the
    free-electron trial, whose number is the Fermi-Dirac sum and whose energy
    is the Wick local energy of its diagonal density matrix."""
    s = cfg1()
    E, N = ed.mixed_estimate(s, s.beta, 0.0)
    E_gc, N_gc = ed.grand_canonical(s)
    assert abs(E - E_gc) < 1e-10 and abs(N - N_gc) < 1e-10
    E0, N0 = ed.mixed_estimate(s, 0.0, s.beta)
    f = fermi_dirac(s.eps, s.mu_T, s.beta)
    assert abs(N0 - 2 * f.sum()) < 1e-10
    E_wick, N_wick = afqmc.local_energy(s, np.diag(1.0 - f).astype(np.complex128))
    assert abs(E0 - E_wick) < 1e-10 and abs(N0 - N_wick) < 1e-10


def _jk(w, O, nb=20):
    idx = np.array_split(np.arange(len(w)), nb)
    full = (np.sum(w * O) / np.sum(w)).real
    jk = np.array([(np.sum(np.delete(w, b) * np.delete(O, b)) / np.sum(np.delete(w, b))).real for b in idx])
    return full, math.sqrt((nb - 1) / nb * np.sum((jk - jk.mean()) ** 2))


@pytest.mark.slow
def test_free_projection_slice_estimates_match_exact_mixed_estimates():
    """Unconstrained walkers, every slice of the N=2, M=7 path: the global
    estimate at slice k against the exact mixed estimate at k (within
    3 sigma plus the Trotter allowance of the tau = beta pin), and the
    slice average against the average of the exact values."""
    s = cfg1()
    n = s.n_slices
    W = 1000
    f = gaussian_fields(7, n, W, s.N_alpha)
    ks, Ek, Nk, Ea, Na, rows = afqmc.slice_estimates(s, f, afqmc.Options(constraint="free", green="two_sided"),
                                                     per_walker=True)
    assert ks == list(range(1, n + 1))
    exact = [ed.mixed_estimate(s, k * s.dtau, (n - k) * s.dtau) for k in ks]
    for k, (w, EL, NL), (Ex, Nx) in zip(ks, rows, exact):
        E, eE = _jk(w, EL)
        Nn, eN = _jk(w, NL)
        assert abs(E - Ex.real) < 3 * eE + 5e-3, (k, E, eE, Ex)
        assert abs(Nn - Nx.real) < 3 * eN + 2e-3, (k, Nn, eN, Nx)
    # the average over slices (its error is at most the largest per-slice error)
    Ex_avg = np.mean([e.real for e, _ in exact])
    Nx_avg = np.mean([x.real for _, x in exact])
    eE_max = max(_jk(w, EL)[1] for w, EL, _ in rows)
    eN_max = max(_jk(w, NL)[1] for w, _, NL in rows)
    assert abs(Ea - Ex_avg) < 3 * eE_max + 5e-3
    assert abs(Na - Nx_avg) < 3 * eN_max + 2e-3
    # a slice estimate differs from the tau = beta one (the average is not trivial)
    assert abs(Ex_avg - exact[-1][0].real) > 0.05


@pytest.mark.slow
def test_planted_trial_block_fails_the_slice_pin(monkeypatch):
    """Planted: the trial block B_T^n at every slice (the power of the
    modified overlap) in the slice estimates of the plain path moves the
    estimate at mid path away from the exact mixed value."""
    s = cfg1()
    n = s.n_slices
    W = 400
    f = gaussian_fields(7, n, W, s.N_alpha)
    good = afqmc.left_diagonal
    monkeypatch.setattr(afqmc, "left_diagonal", lambda sys, k: good(sys, 0))
    ks, Ek, Nk, Ea, Na, rows = afqmc.slice_estimates(s, f[:, :, :], afqmc.Options(constraint="free",
                                                                                  green="two_sided"),
                                                     every=11, per_walker=True)
    k = ks[0]
    Ex, Nx = ed.mixed_estimate(s, k * s.dtau, (n - k) * s.dtau)
    w, EL, NL = rows[0]
    Nn, eN = _jk(w, NL)
    assert abs(Nn - Nx.real) > 3 * eN + 2e-3


def test_slice_estimates_every_and_tau_beta():
    """Recording every 11th slice keeps slices 11 and 22; the last recorded
    estimate equals the weighted estimate at tau = beta."""
    s = cfg1()
    W = 8
    f = gaussian_fields(3, s.n_slices, W, s.N_alpha)
    ks, Ek, Nk, Ea, Na = afqmc.slice_estimates(s, f, every=11)
    assert ks == [11, 22]
    E, N, _ = afqmc.weighted_estimate(afqmc.run(s, f))
    assert abs(Ek[-1].real - E) < 1e-12 and abs(Nk[-1].real - N) < 1e-12
    assert abs(Ea - 0.5 * (Ek[0].real + Ek[1].real)) < 1e-14
