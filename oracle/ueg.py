"""UEG model setup for the oracle (test infrastructure only; see oracle/__init__).

Follows the paper's "Uniform Electron Gas" section (kinetic operator, V_ee,
Madelung term, the sum-of-squares HS form with A(Q), B(Q) and rho(Q)) and the
"Computational Details" section (box length, Fermi temperature, FE trial).

Conventions (shared with the CUDA library only as written conventions, not
as code):

* basis: integer vectors n with |n|^2 <= ncut2, K = 2 pi n / L, ordered by
  (|n|^2, nx, ny, nz) ascending.  M must be a closed-shell count.
* momentum transfers: every nonzero difference n_K' - n_K of two basis
  vectors.  The "half space" is the set whose first nonzero component is
  positive; it is ordered by (|n_Q|^2, nx, ny, nz).  Field alpha = 2q is the
  A field and alpha = 2q+1 the B field of half-space transfer q, so
  N_alpha = N_Q (the number of all nonzero transfers).
"""
import itertools
import math

import numpy as np

MADELUNG_CONSTANT = 2.837297  # Sec. "Uniform Electron Gas", E_M


def closed_shell_cutoff(M):
    """Return ncut2 such that #{n in Z^3 : |n|^2 <= ncut2} == M, else raise."""
    count = 0
    ncut2 = 0
    while count < M:
        r = int(math.isqrt(ncut2)) + 1
        count = sum(1 for n in itertools.product(range(-r, r + 1), repeat=3)
                    if n[0] * n[0] + n[1] * n[1] + n[2] * n[2] <= ncut2)
        if count == M:
            return ncut2
        ncut2 += 1
    raise ValueError(f"M={M} is not a closed-shell plane-wave count")


def basis_integer_vectors(M):
    """Integer plane-wave vectors of the closed shell with M members, in the
    (|n|^2, nx, ny, nz) order.  Sec. "Uniform Electron Gas" (plane-wave basis
    truncated by the kinetic cutoff E_cut)."""
    ncut2 = closed_shell_cutoff(M)
    r = int(math.isqrt(ncut2))
    vecs = [n for n in itertools.product(range(-r, r + 1), repeat=3)
            if n[0] * n[0] + n[1] * n[1] + n[2] * n[2] <= ncut2]
    vecs.sort(key=lambda n: (n[0] * n[0] + n[1] * n[1] + n[2] * n[2], n[0], n[1], n[2]))
    return np.array(vecs, dtype=np.int64)


def box_length(N, rs):
    """L = (4 pi N / 3)^(1/3) r_s  (Computational Details)."""
    return (4.0 * math.pi * N / 3.0) ** (1.0 / 3.0) * rs


def fermi_temperature(rs):
    """k_B T_F = 1/2 (9 pi / 4)^(2/3) / r_s^2  (Eq. fermiT)."""
    return 0.5 * (9.0 * math.pi / 4.0) ** (2.0 / 3.0) / rs ** 2


def fermi_dirac(e, mu, beta):
    """1 / (1 + exp(beta (e - mu))), written to avoid overflow."""
    x = beta * (np.asarray(e, dtype=np.float64) - mu)
    out = np.empty_like(x)
    pos = x > 0
    ex = np.exp(-x[pos])
    out[pos] = ex / (1.0 + ex)
    out[~pos] = 1.0 / (1.0 + np.exp(x[~pos]))
    return out


def _half_space(n):
    for c in n:
        if c != 0:
            return c > 0
    return False


class UEG:
    """All static data of one UEG system.

    Parameters follow the paper: N (target electron number, N-bar), M (basis
    size), r_s, Theta = T / T_F, dtau (requested), mu (None -> mu_T).

    Readings (paper silent / ambiguous):
      * n = round(beta / dtau) slices and dtau := beta / n so that beta is
        exact (Sec. "General formalisms": dtau = beta / n).
      * the Madelung constant enters as E_M = 1/2 * N-bar * xi with
        xi = -2.837297 / L, i.e. half the printed expression; this is the
        value with which the printed N=2, M=7, r_s=3 FCI energy is reproduced
        (tests/golden/fci_n2_m7_rs3.txt).  It uses N-bar, not the sector N.
      * the HS sum of squares equals V_ee plus a one-body term; the
        propagator therefore uses H_1 = T + delta_eps (see one_body_correction).
    """

    def __init__(self, N, M, rs, theta, dtau, mu=None, interacting=True):
        self.interacting = bool(interacting)
        self.N = int(N)
        self.M = int(M)
        self.rs = float(rs)
        self.theta = float(theta)
        self.nvec = basis_integer_vectors(M)
        self.L = box_length(N, rs)
        self.Omega = self.L ** 3
        self.kvec = (2.0 * math.pi / self.L) * self.nvec.astype(np.float64)
        self.eps = 0.5 * np.sum(self.kvec ** 2, axis=1)           # |K|^2 / 2
        self.TF = fermi_temperature(rs)
        self.beta = 1.0 / (theta * self.TF)
        self.n_slices = max(1, int(round(self.beta / dtau)))
        self.dtau = self.beta / self.n_slices
        self._build_transfers()
        self.delta_eps = self.one_body_correction()
        self.mu_T = self.trial_chemical_potential()
        self.mu = self.mu_T if mu is None else float(mu)
        self.E_M = 0.5 * self.N * (-MADELUNG_CONSTANT / self.L)

    # ------------------------------------------------------------------ Q set
    def _build_transfers(self):
        """Momentum transfers Q = K' - K != 0 between basis members.

        Sec. "Uniform Electron Gas": rho(Q) = sum_K a+_{K+Q} a_K with both K and
        K+Q inside the cutoff (the printed a+ a+ is read as a+ a)."""
        index = {tuple(n): i for i, n in enumerate(self.nvec)}
        self.basis_index = index
        qs = set()
        for a in self.nvec:
            for b in self.nvec:
                d = tuple(int(x) for x in (a - b))
                if d != (0, 0, 0):
                    qs.add(d)
        half = sorted([q for q in qs if _half_space(q)],
                      key=lambda n: (n[0] ** 2 + n[1] ** 2 + n[2] ** 2, n[0], n[1], n[2]))
        self.q_half = np.array(half, dtype=np.int64)              # (NQ/2, 3)
        self.NQ = len(qs)
        assert self.NQ == 2 * len(half)
        self.N_alpha = self.NQ
        self.q_half_index = {q: i for i, q in enumerate(half)}
        qk = (2.0 * math.pi / self.L) * self.q_half.astype(np.float64)
        self.q2_half = np.sum(qk ** 2, axis=1)
        # v(Q) = 4 pi / (Omega Q^2); c_Q = sqrt(2 pi / (Omega Q^2))   (A(Q), B(Q))
        self.vq_half = 4.0 * math.pi / (self.Omega * self.q2_half)
        self.cq_half = np.sqrt(2.0 * math.pi / (self.Omega * self.q2_half))
        if not self.interacting:            # non-interacting limit: v(Q) = 0
            self.vq_half = np.zeros_like(self.vq_half)
            self.cq_half = np.zeros_like(self.cq_half)
        # pair lists: for half-space q, the (K', K) with K' - K = +q and = -q
        plus = [[] for _ in half]
        minus = [[] for _ in half]
        for i, a in enumerate(self.nvec):
            for j, b in enumerate(self.nvec):
                if i == j:
                    continue
                d = tuple(int(x) for x in (a - b))
                if d in self.q_half_index:
                    plus[self.q_half_index[d]].append((i, j))
                else:
                    m = tuple(-x for x in d)
                    minus[self.q_half_index[m]].append((i, j))
        self.pairs_plus = [np.array(p, dtype=np.int64).reshape(-1, 2) for p in plus]
        self.pairs_minus = [np.array(p, dtype=np.int64).reshape(-1, 2) for p in minus]

    def one_body_correction(self):
        """delta_eps_K = -(1/(2 Omega)) sum_{Q != 0, K-Q in basis} 4 pi / Q^2.

        Expanding 1/4 sum_Q [A(Q)^2 + B(Q)^2] = (1/(2 Omega)) sum_Q v_Q
        rho(Q) rho(-Q) gives V_ee of the paper plus the one-body operator
        (1/(2 Omega)) sum_Q v_Q sum_{K: K, K-Q in basis} n_K.  The propagator's
        one-body part must subtract it (reading of Eq. for V_ee vs the sum of
        squares; the paper does not print this term)."""
        M = self.M
        out = np.zeros(M)
        if not self.interacting:
            return out
        for i in range(M):
            for j in range(M):
                if i == j:
                    continue
                q = (2.0 * math.pi / self.L) * (self.nvec[i] - self.nvec[j])
                out[i] -= 0.5 * 4.0 * math.pi / (self.Omega * float(q @ q))
        return out

    def trial_chemical_potential(self):
        """mu_T such that 2 sum_K f_FD(eps_K; mu_T, beta) = N-bar (bisection).

        Computational Details: FE trial with <N>_T = N-bar."""
        lo = float(np.min(self.eps)) - 50.0 / self.beta - 10.0
        hi = float(np.max(self.eps)) + 50.0 / self.beta + 10.0
        target = float(self.N)
        if not (0 < target < 2 * self.M):
            raise ValueError("N-bar must lie strictly between 0 and 2M")
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            n = 2.0 * float(np.sum(fermi_dirac(self.eps, mid, self.beta)))
            if n < target:
                lo = mid
            else:
                hi = mid
        return 0.5 * (lo + hi)

    # --------------------------------------------------------------- helpers
    def trial_diagonal(self):
        """(B_T)_KK = exp(-dtau (|K|^2/2 - mu_T))   (Sec. Results, FE trial)."""
        return np.exp(-self.dtau * (self.eps - self.mu_T))

    def kinetic_half_step(self):
        """exp(-dtau/2 (eps_K + delta_eps_K - mu)) for the symmetric Trotter B."""
        return np.exp(-0.5 * self.dtau * (self.eps + self.delta_eps - self.mu))
