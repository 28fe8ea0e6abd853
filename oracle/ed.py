"""Exact diagonalisation of the UEG in a tiny plane-wave basis (oracle; test
infrastructure only).

The Hamiltonian is the paper's H = T + V_ee + E_M (Sec. "Uniform Electron
Gas"), with V_ee in its normal-ordered two-body form

    V_ee = 1/(2 Omega) sum_{Q != 0, K1, K2, s, s'} 4 pi / Q^2
           a+_{K1+Q,s} a+_{K2-Q,s'} a_{K2,s'} a_{K1,s},

every momentum inside the basis.  The grand-canonical ensemble
Z = tr exp(-beta (H - mu N)) (Eq. Z) is summed exactly over the Fock space
of 2M spin-orbitals by blocks of (N_up, N_down, K_total).  This plays the role
of the paper's FT-FCI reference (the paper used HANDE; this is our own code).

Spin-orbital index: p = s * M + k (s = 0 up, 1 down).  A Fock state is a bit
string with bit p set when p is occupied; fermionic signs follow the
convention that operators act on the ordered product of creators with
increasing p.
"""
import math

import numpy as np
import scipy.sparse as sp

from .ueg import UEG


def _popcount(x):
    x = np.asarray(x, dtype=np.int64)
    c = np.zeros_like(x)
    y = x.copy()
    while np.any(y):
        c += y & 1
        y >>= 1
    return c


def _annihilate(states, amp, p):
    """Apply a_p to every state in `states` (vectorised); drop vanishing ones."""
    bit = np.int64(1) << np.int64(p)
    ok = (states & bit) != 0
    s = states[ok]
    a = amp[ok]
    sign = 1 - 2 * (_popcount(s & (bit - 1)) & 1)
    return s ^ bit, a * sign, ok


def _create(states, amp, p):
    bit = np.int64(1) << np.int64(p)
    ok = (states & bit) == 0
    s = states[ok]
    a = amp[ok]
    sign = 1 - 2 * (_popcount(s & (bit - 1)) & 1)
    return s | bit, a * sign, ok


def hamiltonian(sys: UEG, interacting=True):
    """Sparse many-body H - E_M over the full Fock space (2^(2M) states).

    Returns (H csr, occupation numbers N per state, K_total key per state,
    N_up, N_down)."""
    M = sys.M
    if M > 7:
        raise ValueError("exact diagonalisation is only meant for M <= 7")
    nso = 2 * M
    dim = 1 << nso
    states = np.arange(dim, dtype=np.int64)
    rows, cols, vals = [], [], []
    # one-body kinetic energy (diagonal): sum_{k,s} |K|^2/2 n_{k,s}
    diag = np.zeros(dim)
    for s in range(2):
        for k in range(M):
            p = s * M + k
            diag += sys.eps[k] * ((states >> p) & 1)
    rows.append(states)
    cols.append(states)
    vals.append(diag)
    if interacting:
        nvec = sys.nvec
        index = sys.basis_index
        for i1, k1 in enumerate(nvec):          # a_{K1}
            for i2, k2 in enumerate(nvec):      # a_{K2}
                for iq, kq in enumerate(nvec):  # target K1 + Q, enumerate via basis
                    q = kq - k1
                    if not np.any(q):
                        continue
                    t2 = tuple(int(x) for x in (k2 - q))
                    if t2 not in index:
                        continue
                    i4 = index[t2]                       # K2 - Q
                    qq = (2.0 * math.pi / sys.L) * q.astype(np.float64)
                    coef = 0.5 / sys.Omega * 4.0 * math.pi / float(qq @ qq)
                    for s1 in range(2):
                        for s2 in range(2):
                            st = states
                            amp = np.ones(dim)
                            st, amp, ok = _annihilate(st, amp, s1 * M + i1)
                            src = states[ok]
                            st, amp, ok = _annihilate(st, amp, s2 * M + i2)
                            src = src[ok]
                            st, amp, ok = _create(st, amp, s2 * M + i4)
                            src = src[ok]
                            st, amp, ok = _create(st, amp, s1 * M + iq)
                            src = src[ok]
                            if st.size == 0:
                                continue
                            rows.append(st)
                            cols.append(src)
                            vals.append(coef * amp)
    H = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(dim, dim)).tocsr()
    H.sum_duplicates()
    up_mask = (1 << M) - 1
    n_up = _popcount(states & up_mask)
    n_dn = _popcount(states >> M)
    ktot = np.zeros((dim, 3), dtype=np.int64)
    for s in range(2):
        for k in range(M):
            occ = (states >> (s * M + k)) & 1
            ktot += occ[:, None] * sys.nvec[k][None, :]
    return H, n_up, n_dn, ktot


def sector_spectra(sys: UEG, interacting=True):
    """Eigenvalues (without E_M) of every (N_up, N_down, K_total) block.

    Returns a list of (N_up, N_down, K_total tuple, eigenvalues)."""
    H, n_up, n_dn, ktot = hamiltonian(sys, interacting)
    keys = np.concatenate([n_up[:, None], n_dn[:, None], ktot], axis=1)
    _, inverse = np.unique(keys, axis=0, return_inverse=True)
    inverse = inverse.reshape(-1)
    out = []
    order = np.argsort(inverse, kind="stable")
    bounds = np.flatnonzero(np.diff(inverse[order])) + 1
    for idx in np.split(order, bounds):
        block = H[idx][:, idx].toarray()
        if not np.allclose(block, block.conj().T, atol=1e-12):
            raise AssertionError("many-body H block is not Hermitian")
        ev = np.linalg.eigvalsh(0.5 * (block + block.conj().T))
        key = keys[idx[0]]
        out.append((int(key[0]), int(key[1]), tuple(int(x) for x in key[2:]), ev))
    return out


def ground_state_energy(sys: UEG, n_up, n_dn, ktot=(0, 0, 0), interacting=True):
    """Lowest eigenvalue of H (including E_M) in one sector (T = 0 FCI)."""
    best = None
    for nu, nd, kt, ev in sector_spectra(sys, interacting):
        if nu == n_up and nd == n_dn and kt == tuple(ktot):
            best = float(ev[0])
    if best is None:
        raise ValueError("empty sector")
    return best + sys.E_M


def grand_canonical(sys: UEG, beta=None, mu=None, interacting=True):
    """Exact <E> (including E_M) and <N> of exp(-beta (H - mu N)) / Z (Eq. Z,
    thermal average of the paper's Theory section)."""
    beta = sys.beta if beta is None else beta
    mu = sys.mu if mu is None else mu
    energies, numbers = [], []
    for nu, nd, _, ev in sector_spectra(sys, interacting):
        energies.append(ev)
        numbers.append(np.full(ev.shape, nu + nd, dtype=np.float64))
    E = np.concatenate(energies)
    Nn = np.concatenate(numbers)
    x = -beta * (E - mu * Nn)
    x -= x.max()
    w = np.exp(x)
    Z = w.sum()
    return float((w * E).sum() / Z) + sys.E_M, float((w * Nn).sum() / Z)


def one_body_operator(M, X):
    """Fock-space matrix of sum_s sum_ij X_ij a+_{i,s} a_{j,s} (both spins
    carry the same M x M block X)."""
    nso = 2 * M
    dim = 1 << nso
    states = np.arange(dim, dtype=np.int64)
    rows, cols, vals = [], [], []
    for s in range(2):
        for i in range(M):
            for j in range(M):
                if X[i, j] == 0:
                    continue
                st, amp, ok = _annihilate(states, np.ones(dim), s * M + j)
                src = states[ok]
                st, amp, ok = _create(st, amp, s * M + i)
                src = src[ok]
                if st.size:
                    rows.append(st)
                    cols.append(src)
                    vals.append(X[i, j] * amp)
    if not rows:
        return sp.csr_matrix((dim, dim), dtype=np.complex128)
    return sp.coo_matrix((np.concatenate(vals).astype(np.complex128),
                          (np.concatenate(rows), np.concatenate(cols))),
                         shape=(dim, dim)).tocsr()


def number_operator_diagonal(M):
    """N = sum_p n_p on every Fock state, plus (N_up, N_down) labels."""
    states = np.arange(1 << (2 * M), dtype=np.int64)
    up = _popcount(states & ((1 << M) - 1))
    dn = _popcount(states >> M)
    return up + dn, up, dn


def gaussian_state_average(M, X, ops):
    """tr(exp(X^) O) / tr(exp(X^)) for each Fock matrix O in `ops`, and
    ln tr(exp(X^)), where X^ = sum_s sum_ij X_ij a+_is a_js.

    exp(X^) is block diagonal in (N_up, N_down); each block is exponentiated
    densely (scipy expm).  This is the exact many-body trace that the
    generalised Wick theorem reduces to G = (I + e^X)^-1 (Eq. green)."""
    import scipy.linalg as sla
    Xh = one_body_operator(M, X)
    _, up, dn = number_operator_diagonal(M)
    key = up * (2 * M + 1) + dn
    order = np.argsort(key, kind="stable")
    bounds = np.flatnonzero(np.diff(key[order])) + 1
    traces = np.zeros(len(ops), dtype=np.complex128)
    Z = 0.0 + 0.0j
    for idx in np.split(order, bounds):
        U = sla.expm(Xh[idx][:, idx].toarray())
        Z += np.trace(U)
        for n, O in enumerate(ops):
            traces[n] += np.sum(U * O[idx][:, idx].toarray().T)
    return traces / Z, np.log(Z)


def mixed_estimate(sys: UEG, a, b, mu=None, interacting=True):
    """Exact <O> = tr(e^{-a (H - mu N)} e^{-b H_T} O) / tr(e^{-a (H - mu N)} e^{-b H_T})
    for O = H (including E_M) and O = N, with the free-electron trial
    H_T = sum_{k,s} (|K|^2/2 - mu_T) n_{k,s} (Eq. Abrenda with the FE trial of
    Computational Details).  This is what the estimator at tau_k = k dtau
    approaches without a constraint: the walkers' propagators average to
    e^{-k dtau (H - mu N)} and the trial block B_T^(n-k) follows them
    (reading P), so a = k dtau and b = (n - k) dtau.  Returns complex values
    (the two factors do not commute)."""
    mu = sys.mu if mu is None else mu
    H, n_up, n_dn, ktot = hamiltonian(sys, interacting)
    dim = H.shape[0]
    states = np.arange(dim, dtype=np.int64)
    ht = np.zeros(dim)
    for s in range(2):
        for k in range(sys.M):
            ht += (sys.eps[k] - sys.mu_T) * ((states >> (s * sys.M + k)) & 1)
    nn = (n_up + n_dn).astype(np.float64)
    keys = np.concatenate([n_up[:, None], n_dn[:, None], ktot], axis=1)
    _, inverse = np.unique(keys, axis=0, return_inverse=True)
    inverse = inverse.reshape(-1)
    order = np.argsort(inverse, kind="stable")
    bounds = np.flatnonzero(np.diff(inverse[order])) + 1
    blocks = []
    shift = None
    for idx in np.split(order, bounds):
        h = H[idx][:, idx].toarray()
        ev, V = np.linalg.eigh(0.5 * (h + h.conj().T))
        x = -a * (ev - mu * nn[idx[0]])
        y = -b * ht[idx]
        m = x.max() + y.max()
        shift = m if shift is None else max(shift, m)
        blocks.append((idx, h, ev, V, x, y))
    Z = E = Nn = 0j
    for idx, h, ev, V, x, y in blocks:
        # e^{-a (H - mu N)} e^{-b H_T} on this block, scaled by e^{-shift}
        U = (V * np.exp(x - 0.5 * shift)[None, :]) @ V.conj().T
        U = U * np.exp(y - 0.5 * shift)[None, :]
        Z += np.trace(U)
        E += np.sum(U * h.T)
        Nn += np.trace(U) * nn[idx[0]]
    return E / Z + sys.E_M, Nn / Z
