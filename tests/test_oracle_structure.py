"""Pins of the oracle's density correlation <rho(Q) rho(-Q)> (the numerator
of the static structure factor): the exact Fock-space trace tr(U rho rho)/tr U
for a random one-body U = exp(X) (both spins), the free-fermion closed form
2 sum_K f_{K+Q} (1 - f_K) for a diagonal density matrix, and a planted
mistake (the anticommutator term dropped) that the Fock pin catches."""
import numpy as np
import scipy.linalg as sla

from oracle import afqmc, ed
from oracle.ueg import UEG


def cfg1():
    return UEG(2, 7, 1.0, 0.5, 0.05)


def rho_matrix(s, qvec):
    """One spin block of rho(Q): X[i, j] = 1 when n_i - n_j = Q (both in the basis)."""
    n = s.nvec
    X = np.zeros((s.M, s.M))
    for i in range(s.M):
        for j in range(s.M):
            if np.array_equal(n[i] - n[j], qvec):
                X[i, j] = 1.0
    return X


def test_matches_fock_space_trace():
    s = cfg1()
    rng = np.random.default_rng(8)
    X = 0.4 * (rng.standard_normal((7, 7)) + 1j * rng.standard_normal((7, 7))) - np.diag(s.eps - 1.0)
    G = np.linalg.inv(np.eye(7) + sla.expm(X))
    plus, minus = afqmc.density_correlation(s, G)
    ops, want = [], []
    for q in range(len(s.q_half)):
        for sgn, val in ((1, plus[q]), (-1, minus[q])):
            qv = sgn * np.asarray(s.q_half[q])
            A = ed.one_body_operator(s.M, rho_matrix(s, qv))
            B = ed.one_body_operator(s.M, rho_matrix(s, -qv))
            ops.append(A @ B)
            want.append(val)
    avg, _ = ed.gaussian_state_average(s.M, X, ops)
    assert np.max(np.abs(avg - np.array(want))) < 1e-10 * max(1.0, np.max(np.abs(avg)))


def test_free_fermion_closed_form():
    s = UEG(14, 57, 1.0, 0.125, 0.05)
    f = 1.0 / (1.0 + np.exp(s.beta * (s.eps - s.mu)))
    G = np.diag(1.0 - f).astype(np.complex128)          # P = diag(f)
    plus, minus = afqmc.density_correlation(s, G)
    n = s.nvec
    index = {tuple(v): i for i, v in enumerate(n)}
    for q in range(len(s.q_half)):
        for sgn, val in ((1, plus[q]), (-1, minus[q])):
            qv = sgn * np.asarray(s.q_half[q])
            ref = 0.0
            for k in range(s.M):
                kq = index.get(tuple(n[k] + qv))
                if kq is not None:
                    ref += 2.0 * f[kq] * (1.0 - f[k])
            assert abs(val - ref) < 1e-12 * max(1.0, ref)


def test_planted_missing_anticommutator_term_is_caught(monkeypatch):
    s = cfg1()
    rng = np.random.default_rng(8)
    X = 0.4 * (rng.standard_normal((7, 7)) + 1j * rng.standard_normal((7, 7))) - np.diag(s.eps - 1.0)
    G = np.linalg.inv(np.eye(7) + sla.expm(X))
    qv = np.asarray(s.q_half[0])
    A = ed.one_body_operator(s.M, rho_matrix(s, qv))
    B = ed.one_body_operator(s.M, rho_matrix(s, -qv))
    (exact,), _ = ed.gaussian_state_average(s.M, X, [A @ B])
    good = afqmc.density_correlation(s, G)[0][0]
    assert abs(good - exact) < 1e-10
    P = afqmc.one_rdm(G)
    dq = 2.0 * np.sum(P[s.pairs_plus[0][:, 0], s.pairs_plus[0][:, 0]])
    assert abs((good - dq) - exact) > 1e-3
