"""Phaseless finite-temperature AFQMC walker propagation for the UEG
(oracle; test infrastructure only, see oracle/__init__).

Plain complex128 NumPy/SciPy, one walker at a time, following the paper's
Theory section (Eqs. B, HS, grand2, green, Abrenda, ftoratio, import,
phimport, theta), "Numerical Stabilization" (QRCP / QDT and the stable G),
"Exploiting the stack structure", and the UEG local energy (E_1, E_2 with
Gamma_Q and Lambda_Q).

Readings where the paper is silent, garbled or inconsistent:

A  HS sign vs force bias.  The paper writes exp(-sqrt(dtau) x.v) but its
   force bias xbar = -sqrt(dtau)(<v> - v0) cancels the O(sqrt(dtau)) term only
   for exp(+sqrt(dtau) x.v).  We propagate with exp(+sqrt(dtau)(x - xbar).v)
   and xbar = -sqrt(dtau) <v>.  (Pinned: d ln I / dx at x = 0 is O(dtau).)
B  rho(Q) = sum_K a+_{K+Q} a_K (the printed a+ a+ is a misprint).  The HS
   operators are v_A(Q) = i A(Q), v_B(Q) = i B(Q) for Q in the half space,
   so H_2 = -1/2 sum v^2.  Per spin the one-body matrix of y.v is
   V_{K+Q,K} = sqrt(dtau) c_Q i (y_A + i y_B), V_{K-Q,K} = sqrt(dtau) c_Q i
   (y_A - i y_B), zero diagonal.  (Pinned: anti-Hermitian for real y.)
C  The sum of squares carries an extra one-body term; the propagator uses
   H_1 = T + delta_eps (oracle.ueg.UEG.one_body_correction).  The FE trial
   stays the bare |K|^2/2 - mu_T.
D  Spin: fields couple to the spin-summed density, so both spin blocks of
   B are the same M x M matrix; one chain per walker, S_k = (per-spin
   ratio)^2, <rho(Q)> = 2 rho-bar_Q, N = 2 tr P, E_1 doubled, exchange
   same-spin only.
E  Gamma_Q (garbled in print) = <rho(Q)><rho(-Q)>; Lambda_Q = sum_s sum_{K1,K2}
   P_{K1+Q,K2} P_{K2-Q,K1} with every index in the basis.
F  The printed stable-G formula transposes the wrong factors; the
   derivation that follows it gives G = T^-1 (D_b Q^H T^-1 + D_s)^-1 D_b Q^H
   (Q^T read as Q^H for complex matrices, sgn(D) = D/|D|).
I  exp(V) is a Taylor series of order p (default 6); Pade expm is reported
   beside it as the truncation error.
K  theta_k = arg S_k evaluated on the shifted fields; a walker with
   cos(theta_k) <= 0 is killed (weight 0) and stays dead, and so is a walker
   whose ratio or Gaussian factor is not finite (the paper is silent there).
L  Estimates are taken at tau = beta; sum_w w Re(eps) / sum_w w.
M  B uses mu, B_T uses mu_T.

P  P(tau) in the optimal force bias is the equal-time one-body density
   matrix at tau, P = I - G(tau)^T with G(tau) = (I + R D_L)^-1: the
   propagated block R (slices 1..k) with the trial block D_L = B_T^(n-k)
   (slices k+1..n) placed cyclically after it.  Only this G cancels the
   O(sqrt(dtau)) term of ln I_k (pinned by a finite-difference test; with
   (I + D_L R)^-1, the tau = beta form of Eq. green, the gradient is as large
   as with no force bias).  At tau = beta both forms coincide, so the
   estimators are unchanged.

S  Modified overlap ratio (Eq. ztfix; proposed in the T -> 0 discussion, not
   evaluated there).  With Options(overlap="modified") the trial block is
   B_T^n at every slice, A~_k = B_T^n B_k ... B_1, and the weight uses
   S~_k = [det(I + A~_k) / det(I + A~_{k-1})]^2 in place of S_k (theta_k =
   arg S~_k); the force bias is the optimal one for S~ (reading P with
   D_L = B_T^n).  The target stays the physical ensemble: after slice n the
   estimators use G(beta) = (I + R_n)^-1 and the weight takes one more ratio
   r = [det(I + R_n) / det(I + B_T^n R_n)]^2, projected like a slice ratio
   (|r| max(0, cos arg r) phaseless, r in free projection), with no Gaussian
   factor.  In free projection with no force bias the final weight equals
   the Eq. ftoratio one exactly (both telescope to the same determinants).

T  Low-rank truncation (Sec. "Exploiting the low-rank structure", Eq. thresh;
   threshold absolute, the paper's production value 1e-6).  With
   Options(low_rank=thr) every stabilisation keeps the leading columns of the
   pivoted QR whose |R_jj| >= thr (Businger-Golub pivoting makes |R_jj|
   non-increasing, so Eq. thresh keeps a prefix; at least one), so the right
   block is R = Y d_R t_R with Y M x m, t_R m x M.  The left block D_L keeps
   the entries >= thr (m_L of them).  G(tau) = (I + R D_L)^-1 follows the
   paper's steps in the cyclic order of reading P: core c = d_R t_R[:, L] d_L
   (m x m_L), its QRCP c = q_c r_c pi_c, q = Y q_c, d = diag r_c,
   t = (d^-1 r_c)(pi_c P_L^T); then Woodbury and the determinant lemma in
   m_T = min(m, m_L) dimensions with the scales of d split as in the stable
   G: I + d t q = d_b^-1 (d_b + d_s X), X = t q, so
   G = I - q (d_b + d_s X)^-1 d_s t and ln det(I + A) = ln det(d_b + d_s X)
   - sum ln d_b (the paper splits the same product on the other side of X,
   (X^-1 d_b + d_s) d_b^-1 X; the two are equal and ours needs no X^-1).

Slice bookkeeping (Eq. Abrenda): before slice k the right block
R_{k-1} = B_{k-1} ... B_1 is held as Y D T (Y = B's since the last QRCP times
Q_R); the left block is the diagonal D_L = B_T^(n-(k-1)).  Slice k: force
bias from G(tau_{k-1}); B_k from x_k - xbar_k; Y <- B_k Y; QRCP of Y D every
s slices; G(tau_k) and ln det(I + A_k) with D_L = B_T^(n-k); weight update.
"""
import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .ueg import UEG


# ---------------------------------------------------------------- one-body ops
def density_sums(sys: UEG, P):
    """rho-bar_Q = sum_K P_{K+Q,K} for every half-space Q (plus) and for -Q
    (minus).  Sec. "Uniform Electron Gas", rho(Q); P is one spin block."""
    nh = len(sys.pairs_plus)
    rp = np.zeros(nh, dtype=np.complex128)
    rm = np.zeros(nh, dtype=np.complex128)
    for q in range(nh):
        pp = sys.pairs_plus[q]
        pm = sys.pairs_minus[q]
        rp[q] = np.sum(P[pp[:, 0], pp[:, 1]])
        rm[q] = np.sum(P[pm[:, 0], pm[:, 1]])
    return rp, rm


def one_rdm(G):
    """P = I - G^T  (Eq. green and the 1RDM that follows it)."""
    return np.eye(G.shape[0]) - G.T


def force_bias(sys: UEG, G):
    """Optimal force bias xbar_alpha = -sqrt(dtau) (<v_alpha> - v0_alpha).

    <v_A(Q)> = 2 i c_Q (rho_Q + rho_-Q), <v_B(Q)> = -2 c_Q (rho_Q - rho_-Q)
    (factor 2: two identical spin blocks).  The mean-field shift v0 is
    sum_pq v_pq (P_T)_pq, which vanishes because P_T is diagonal and every
    v_alpha has a zero diagonal (Q != 0)."""
    P = one_rdm(G)
    rp, rm = density_sums(sys, P)
    vA = 2j * sys.cq_half * (rp + rm)
    vB = -2.0 * sys.cq_half * (rp - rm)
    xbar = np.empty(sys.N_alpha, dtype=np.complex128)
    xbar[0::2] = -math.sqrt(sys.dtau) * vA
    xbar[1::2] = -math.sqrt(sys.dtau) * vB
    return xbar


def hs_matrix(sys: UEG, y):
    """V = sqrt(dtau) sum_alpha y_alpha v_alpha (one spin block; reading B)."""
    M = sys.M
    V = np.zeros((M, M), dtype=np.complex128)
    yA = y[0::2]
    yB = y[1::2]
    s = math.sqrt(sys.dtau)
    a = s * sys.cq_half * 1j * (yA + 1j * yB)   # coefficient of rho(Q)
    b = s * sys.cq_half * 1j * (yA - 1j * yB)   # coefficient of rho(-Q)
    for q in range(len(sys.pairs_plus)):
        pp = sys.pairs_plus[q]
        pm = sys.pairs_minus[q]
        V[pp[:, 0], pp[:, 1]] = a[q]
        V[pm[:, 0], pm[:, 1]] = b[q]
    return V


def expm_taylor(V, p):
    """sum_{j=0..p} V^j / j!  (reading I)."""
    E = np.eye(V.shape[0], dtype=np.complex128)
    term = np.eye(V.shape[0], dtype=np.complex128)
    for j in range(1, p + 1):
        term = term @ V / j
        E = E + term
    return E


def propagator(sys: UEG, y, p, exact_exp=False):
    """B = exp(-dtau/2 K~) exp(V(y)) exp(-dtau/2 K~), K~ = eps + delta_eps - mu
    (Eq. B with the symmetric Trotter split; readings A-C)."""
    h = sys.kinetic_half_step()
    V = hs_matrix(sys, y)
    E = sla.expm(V) if exact_exp else expm_taylor(V, p)
    return h[:, None] * E * h[None, :]


def left_diagonal(sys: UEG, k):
    """Diagonal of B_T^(n-k) (Eq. Abrenda, FE trial)."""
    return np.exp(-(sys.n_slices - k) * sys.dtau * (sys.eps - sys.mu_T))


# ---------------------------------------------------------------- QRCP / UDT
def qrcp(C):
    """Column-pivoted QR C = Q R Pi (Sec. Numerical Stabilization).

    Returns Q, D = diag R, U = D^-1 R (unit upper) and the pivot list piv with
    C[:, piv] = Q R."""
    Q, R, piv = sla.qr(C, pivoting=True)
    D = np.diag(R).copy()
    U = R / D[:, None]
    return Q, D, U, piv


def stabilise(Y, D, T):
    """One stratification step: Y D = Q R Pi, D <- diag R,
    T <- (D^-1 R)(Pi T); the chain restarts from Y = Q."""
    Q, Dn, U, piv = qrcp(Y * D[None, :])
    Tn = U @ T[piv, :]
    return Q, Dn, Tn


def _split(D):
    """D_b, D_s of the stable-G formula (Sec. Numerical Stabilization):
    D_b = 1/|D| if |D| > 1 else 1;  D_s = D if |D| <= 1 else D/|D|."""
    a = np.abs(D)
    big = a > 1.0
    Db = np.where(big, 1.0 / np.where(big, a, 1.0), 1.0)
    Ds = np.where(big, D / np.where(big, a, 1.0), D)
    return Db, Ds


def _clog_det(Mx):
    sign, logabs = np.linalg.slogdet(Mx)
    return logabs + 1j * np.angle(sign)


def green_paper(DL, Y, D, T):
    """G(tau) and ln det(I + A) by stratification and the paper's stable formula.

    The equal-time Green's function at tau = k dtau is G(tau) = (I + R D_L)^-1
    with R = Y D T the propagated block (slices 1..k) and D_L = B_T^(n-k) the
    trial block (slices k+1..n) placed cyclically to its right (reading P of
    the optimal force bias; det(I + R D_L) = det(I + D_L R) = det(I + A(tau))).
    R D_L is brought to QDT form by two stratification steps (QRCP of Y D,
    then of D_CR T_CR D_L), and G = T^-1 (D_b Q^H T^-1 + D_s)^-1 D_b Q^H
    (reading F).  ln det(I + A) = ln det Q - sum ln D_b
    + ln det(D_b Q^H T^-1 + D_s) + ln det T."""
    Q1, D1, U1, p1 = qrcp(Y * D[None, :])
    T1 = U1 @ T[p1, :]
    Q2, Dn, U2, p2 = qrcp(D1[:, None] * T1 * DL[None, :])
    Q = Q1 @ Q2
    Tn = U2[:, np.argsort(p2)]                     # D^-1 R Pi with C[:, p2] = Q R
    Db, Ds = _split(Dn)
    Tinv = np.linalg.inv(Tn)
    M1 = Db[:, None] * (Q.conj().T @ Tinv) + np.diag(Ds)
    G = Tinv @ np.linalg.solve(M1, Db[:, None] * Q.conj().T)
    ld = _clog_det(Q) - np.sum(np.log(Db)) + _clog_det(M1) + _clog_det(Tn)
    return G, ld


def green_two_sided(DL, Y, D, T):
    """G(tau) = (I + Y D T D_L)^-1 and ln det with the scales split on both
    sides of the inner matrix (same derivation as the paper's stable G):

    I + D_L Y D T = D_Lb^-1 Mt D_Rb^-1 T,  Mt = D_Lb T^-1 D_Rb + D_Ls Y D_Rs,
    and by push-through (I + R D_L)^-1 = I - R (I + D_L R)^-1 D_L
                                       = I - Y D_Rs Mt^-1 D_Ls,
    every factor bounded.  ln det(I + A) = -sum ln D_Lb - sum ln D_Rb
    + ln det Mt + ln det T."""
    Lb, Ls = _split(DL.astype(np.complex128))
    Rb, Rs = _split(D)
    Tinv = np.linalg.inv(T)
    Mt = Lb[:, None] * Tinv * Rb[None, :] + Ls[:, None] * Y * Rs[None, :]
    G = np.eye(len(D)) - (Y * Rs[None, :]) @ np.linalg.solve(Mt, np.diag(Ls))
    ld = (-np.sum(np.log(Lb)) - np.sum(np.log(Rb)) + _clog_det(Mt) + _clog_det(T))
    return G, ld


def green_direct(DL, Y, D, T):
    """(I + R D_L)^-1 and ln det(I + R D_L) with R = Y D T formed explicitly
    (only for well-conditioned products)."""
    A = (Y * D[None, :]) @ T * DL[None, :]
    I = np.eye(A.shape[0])
    return np.linalg.inv(I + A), _clog_det(I + A)


GREEN = {"paper": green_paper, "two_sided": green_two_sided, "direct": green_direct}


# ---------------------------------------------------------------- low rank (reading T)
def stabilise_truncated(Y, D, T, thr):
    """Stratification step of the right block followed by Eq. thresh: QRCP of
    Y D (M x m), keep the leading columns with |R_jj| >= thr (at least one).
    Returns Y (M x m'), D (m'), T (m' x M)."""
    Q, R, piv = sla.qr(Y * D[None, :], pivoting=True, mode="economic")
    Dn = np.diag(R).copy()
    Tn = (R / Dn[:, None]) @ T[piv, :]
    small = np.abs(Dn) < thr
    m = int(np.argmax(small)) if small.any() else len(Dn)
    m = max(m, 1)
    return Q[:, :m], Dn[:m], Tn[:m, :]


def left_keep(DL, thr):
    """Indices of the left block entries kept by Eq. thresh (at least the largest)."""
    keep = np.nonzero(DL >= thr)[0]
    return keep if len(keep) else np.array([int(np.argmax(DL))])


def green_lowrank(DL, Y, D, T, thr):
    """G(tau) = (I + R D_L)^-1 and ln det(I + R D_L) with R = Y diag(D) T of rank
    m and D_L truncated by Eq. thresh (Sec. "Exploiting the low-rank
    structure"): core c = D T[:, L] d_L, QRCP c = q_c r_c pi_c, q = Y q_c,
    d = diag r_c, t = (d^-1 r_c)(pi_c P_L^T), X = t q, then the Woodbury
    identity and the matrix determinant lemma in m_T dimensions."""
    M = Y.shape[0]
    L = left_keep(DL, thr)
    c = D[:, None] * T[:, L] * DL[L][None, :]
    Qc, R, piv = sla.qr(c, pivoting=True, mode="economic")
    d = np.diag(R).copy()
    U = R / d[:, None]
    q = Y @ Qc
    t = np.zeros((len(d), M), dtype=np.complex128)
    t[:, L[piv]] = U
    X = t @ q
    Db, Ds = _split(d)
    Mx = np.diag(Db).astype(np.complex128) + Ds[:, None] * X
    G = np.eye(M) - q @ np.linalg.solve(Mx, Ds[:, None] * t)
    ld = _clog_det(Mx) - np.sum(np.log(Db))
    return G, ld


# ---------------------------------------------------------------- estimators
def local_energy(sys: UEG, G):
    """Local energy eps = E_M + E_1 + E_2 and particle number N from
    P = I - G^T (Sec. "Uniform Electron Gas", local energy; readings D, E).

    E_1 = 2 sum_K |K|^2/2 P_KK; E_2 = 1/(2 Omega) sum_{Q != 0} 4 pi/Q^2
    (Gamma_Q - Lambda_Q), Gamma_Q = (2 rho_Q)(2 rho_-Q),
    Lambda_Q = 2 sum_{K1 K2} P_{K1+Q,K2} P_{K2-Q,K1}."""
    P = one_rdm(G)
    Nloc = 2.0 * np.trace(P)
    E1 = 2.0 * np.sum(sys.eps * np.diag(P))
    rp, rm = density_sums(sys, P)
    E2 = 0.0 + 0.0j
    for q in range(len(sys.q_half)):
        for sgn, vq_pairs in ((1, sys.pairs_plus[q]), (-1, sys.pairs_minus[q])):
            gam = (2.0 * rp[q]) * (2.0 * rm[q])      # same for +Q and -Q
            # (a, d) = (K1+Q, K1);  (b, c) = (K2, K2-Q), all four in the basis
            b, c = _shifted_pairs(sys, sgn, q)
            a, d = vq_pairs[:, 0], vq_pairs[:, 1]
            lam = 2.0 * np.sum(P[np.ix_(a, b)] * P[np.ix_(c, d)].T)
            E2 += sys.vq_half[q] / 2.0 * (gam - lam)
    return sys.E_M + E1 + E2, Nloc


def density_correlation(sys: UEG, G):
    """<rho(Q) rho(-Q)> for every Q != 0 from P = I - G^T (Wick's theorem;
    readings B, D, E), the numerator of the static structure factor
    S(Q) = <rho(Q) rho(-Q)> / N (Results, structure factor).

    Contracting a+_{K1+Q} a_K1 a+_{K2-Q} a_K2 gives Gamma_Q (both pairs
    closed), -Lambda_Q (crossed, same spin) and, from the anticommutator
    a_K1 a+_{K2-Q} = delta - a+ a, D_Q = 2 sum_{K: K, K+Q in basis} P_{K+Q,K+Q}.
    Returns (plus, minus): arrays over the half-space q for Q = +q and -q."""
    P = one_rdm(G)
    rp, rm = density_sums(sys, P)
    nh = len(sys.q_half)
    out = {1: np.zeros(nh, np.complex128), -1: np.zeros(nh, np.complex128)}
    for q in range(nh):
        for sgn, pairs in ((1, sys.pairs_plus[q]), (-1, sys.pairs_minus[q])):
            gam = (2.0 * rp[q]) * (2.0 * rm[q])
            b, c = _shifted_pairs(sys, sgn, q)
            a, d = pairs[:, 0], pairs[:, 1]                  # (a, d) = (K + Q, K)
            lam = 2.0 * np.sum(P[np.ix_(a, b)] * P[np.ix_(c, d)].T)
            dq = 2.0 * np.sum(P[a, a])
            out[sgn][q] = gam - lam + dq
    return out[1], out[-1]


def _shifted_pairs(sys: UEG, sgn, q):
    """Basis indices (b, c) with n_c = n_b - sgn * q_half[q], both in the basis
    (the pair lists read back in the opposite orientation)."""
    pairs = sys.pairs_plus[q] if sgn > 0 else sys.pairs_minus[q]
    # pairs hold (i, j) with n_i - n_j = sgn * q, so b = i, c = j
    return pairs[:, 0], pairs[:, 1]


# ---------------------------------------------------------------- propagation
@dataclass
class Options:
    stabilise_every: int = 5
    exp_order: int = 6
    constraint: str = "phaseless"      # or "free"
    overlap: str = "paper"             # "paper" (Eq. ftoratio) | "modified" (Eq. ztfix)
    low_rank: float = 0.0              # threshold of Eq. thresh (reading T); 0 = full rank
    green: str = "paper"               # "paper" | "two_sided" | "direct"
    exact_exp: bool = False
    force_bias: bool = True


@dataclass
class WalkerState:
    """Right block Y D T, current G_k, ln det(I + A_k), weight and alive flag."""
    Y: np.ndarray
    D: np.ndarray
    T: np.ndarray
    G: np.ndarray
    logdet: complex
    logw: complex = 0j
    alive: bool = True


@dataclass
class WalkerResult:
    logw: complex
    alive: bool
    G: np.ndarray
    logdet: complex
    energy: complex
    number: complex
    logdet_trace: list = field(default_factory=list)
    lnS_trace: list = field(default_factory=list)
    xbar_trace: list = field(default_factory=list)
    rank_trace: list = field(default_factory=list)


def initial_state(sys: UEG):
    """A(0) = B_T^n: right block I, G_0 = (I + B_T^n)^-1 (Eq. Abrenda, k = 0)."""
    M = sys.M
    dl = left_diagonal(sys, 0)
    G = np.diag(1.0 / (1.0 + dl)).astype(np.complex128)
    return WalkerState(np.eye(M, dtype=np.complex128), np.ones(M, dtype=np.complex128),
                       np.eye(M, dtype=np.complex128), G, complex(np.sum(np.log1p(dl))))


def update_weight(logw, alive, lnS, gauss, constraint):
    """w <- |I| max(0, cos theta) with I = S e^gauss, theta = arg S (Eqs.
    import, phimport, theta; reading K), or w <- w I in free projection.
    A phaseless walker whose ratio or Gaussian factor is not finite is
    dropped (weight 0; the paper is silent on non-finite ratios)."""
    if constraint == "free":
        return logw + lnS + gauss, alive
    if alive:
        c = math.cos(lnS.imag)                      # theta_k = arg S_k
        if not (math.isfinite(lnS.real + gauss.real) and math.isfinite(c)):
            return logw, False
        if c <= 0.0:
            return logw, False
        return logw + lnS.real + gauss.real + math.log(c), alive
    return logw, alive


def slice_step(sys: UEG, st: WalkerState, x, k, opts: Options, xbar=None):
    """Slice k (1-based) of Eq. Abrenda: force bias from G_{k-1}, B_k from the
    shifted field, Y <- B_k Y, QRCP every s slices, G_k and ln det, then the
    phaseless (Eqs. import, phimport, theta) or free-projection weight.  With
    the modified overlap (Eq. ztfix, reading S) the trial block stays B_T^n
    and slice n ends with the physical G(beta) and the ratio r.

    Returns (new state, lnS_k, gauss_k, xbar_k)."""
    x = np.asarray(x, dtype=np.float64)
    if xbar is None:
        xbar = force_bias(sys, st.G) if opts.force_bias else np.zeros(sys.N_alpha, np.complex128)
    B = propagator(sys, x - xbar, opts.exp_order, opts.exact_exp)
    Y, D, T = B @ st.Y, st.D, st.T
    thr = opts.low_rank
    if opts.stabilise_every > 0 and k % opts.stabilise_every == 0:
        Y, D, T = stabilise_truncated(Y, D, T, thr) if thr > 0 else stabilise(Y, D, T)
    green = (lambda DL, Y, D, T: green_lowrank(DL, Y, D, T, thr)) if thr > 0 else GREEN[opts.green]
    modified = opts.overlap == "modified"
    Gn, ldn = green(left_diagonal(sys, 0 if modified else k), Y, D, T)
    lnS = 2.0 * (ldn - st.logdet)                  # two identical spin blocks
    gauss = np.sum(x * xbar - 0.5 * xbar * xbar)   # Eq. import
    logw, alive = update_weight(st.logw, st.alive, lnS, gauss, opts.constraint)
    if modified and k == sys.n_slices:
        Gp, ldp = green(left_diagonal(sys, k), Y, D, T)
        logw, alive = update_weight(logw, alive, 2.0 * (ldp - ldn), 0j, opts.constraint)
        Gn, ldn = Gp, ldp
    return WalkerState(Y, D, T, Gn, ldn, logw, alive), lnS, gauss, xbar


def propagate_walker(sys: UEG, fields, opts: Options, n_slices=None, record=False,
                     want_estimator=True):
    """Propagate one walker over `n_slices` slices (default: the whole path).

    fields: real array [n_slices, N_alpha] of N(0,1) draws x_k."""
    n = sys.n_slices if n_slices is None else n_slices
    st = initial_state(sys)
    res = WalkerResult(0j, True, st.G, st.logdet, 0j, 0j)
    for k in range(1, n + 1):
        st, lnS, _, xbar = slice_step(sys, st, fields[k - 1], k, opts)
        if record:
            res.logdet_trace.append(st.logdet)
            res.lnS_trace.append(lnS)
            res.xbar_trace.append(xbar)
            res.rank_trace.append(len(st.D))
    res.logw, res.alive, res.G, res.logdet = st.logw, st.alive, st.G, st.logdet
    if want_estimator:
        res.energy, res.number = local_energy(sys, st.G)
    return res


def run(sys: UEG, fields, opts: Options = None, n_slices=None, record=False,
        want_estimator=True):
    """Propagate every walker.  fields: [n_slices, W, N_alpha]."""
    opts = opts or Options()
    W = fields.shape[1]
    return [propagate_walker(sys, fields[:, w, :], opts, n_slices, record, want_estimator)
            for w in range(W)]


def slice_estimates(sys: UEG, fields, opts: Options = None, every=1, per_walker=False):
    """Global estimates E(tau_k), N(tau_k) after every `every`-th slice and
    their average over those slices (Results, "Assessing the Phaseless
    Constraint": "No Average" is the estimate at tau = beta, "Average" the
    global estimate averaged over the time slices).

    All walkers advance together; after slice k the estimate is
    sum_i w_i,k O_L,i,k / sum_i w_i,k with the weights of slice k and the
    local values from G(tau_k) (reading P), real parts taken as in reading L
    (complex weights in free projection).  Reading (the paper gives no
    formula): every recorded slice counts once in the average.
    Returns (ks, E_k, N_k, E_avg, N_avg) with complex E_k, N_k; with
    per_walker=True also a list over the recorded slices of (w, E_L, N_L)
    arrays (the scaled weights and local values of every walker)."""
    opts = opts or Options()
    n, W = fields.shape[0], fields.shape[1]
    states = [initial_state(sys) for _ in range(W)]
    ks, Es, Ns, rows = [], [], [], []
    for k in range(1, n + 1):
        states = [slice_step(sys, st, fields[k - 1, w], k, opts)[0] for w, st in enumerate(states)]
        if k % every:
            continue
        res = [WalkerResult(st.logw, st.alive, st.G, st.logdet, *local_energy(sys, st.G)) for st in states]
        if opts.constraint == "free":
            lw = np.array([r.logw for r in res])
            w = np.exp(lw - np.max(lw.real))
        else:
            ok = np.array([r.alive and math.isfinite(r.logw.real) for r in res])
            lw = np.where(ok, np.array([r.logw.real for r in res]), -np.inf)
            w = np.where(ok, np.exp(lw - np.max(lw)), 0.0)
        EL = np.array([r.energy for r in res])
        NL = np.array([r.number for r in res])
        E = np.sum(w * EL) / np.sum(w)
        Nn = np.sum(w * NL) / np.sum(w)
        if per_walker:
            rows.append((w, EL, NL))
        ks.append(k)
        Es.append(E)
        Ns.append(Nn)
    Es, Ns = np.array(Es), np.array(Ns)
    out = (ks, Es, Ns, float(np.mean(Es.real)), float(np.mean(Ns.real)))
    return out + (rows,) if per_walker else out


def weighted_estimate(results, constraint="phaseless"):
    """<O> = sum_i w_i O_i / sum_i w_i (Theory: importance-sampled estimator).

    Returns (E, N, sum_w) with w scaled by exp(-max ln|w|)."""
    lw = np.array([r.logw for r in results], dtype=np.complex128)
    alive = np.array([r.alive for r in results])
    E = np.array([r.energy for r in results])
    Nn = np.array([r.number for r in results])
    if constraint == "free":
        ref = np.max(lw.real)
        w = np.exp(lw - ref)
        return np.sum(w * E) / np.sum(w), np.sum(w * Nn) / np.sum(w), np.sum(w)
    ok = alive & np.isfinite(lw.real)               # a non-finite ln|w| weighs 0
    lwr = np.where(ok, lw.real, -np.inf)
    ref = np.max(lwr)
    w = np.where(ok, np.exp(lwr - ref), 0.0)
    return np.sum(w * E.real) / np.sum(w), np.sum(w * Nn.real) / np.sum(w), np.sum(w)


# ---------------------------------------------------------------- mu derivative
def _with_mu(sys: UEG, mu):
    """A shallow copy of `sys` whose propagator uses chemical potential mu
    (B_T and mu_T unchanged, reading M)."""
    import copy
    s = copy.copy(sys)
    s.mu = float(mu)
    return s


def path_with_fixed_bias(sys: UEG, fields, opts: Options, xbars):
    """Propagate one walker with the force bias of every slice given
    (xbars[k-1] for slice k) instead of computed from G."""
    st = initial_state(sys)
    for k in range(1, sys.n_slices + 1):
        st, *_ = slice_step(sys, st, fields[k - 1], k, opts, xbar=xbars[k - 1])
    return st


def mu_observables(sys: UEG, fields, opts: Options = None, mu=None, xbars=None):
    """Per-walker (ln w, alive, E_L, N_L) at tau = beta for chemical potential
    mu; with `xbars` ([W][n][N_alpha]) the force bias is held at those values."""
    opts = opts or Options()
    s = sys if mu is None else _with_mu(sys, mu)
    out = []
    for w in range(fields.shape[1]):
        if xbars is None:
            r = propagate_walker(s, fields[:, w, :], opts, record=True)
            out.append((r.logw, r.alive, r.energy, r.number, r.xbar_trace))
        else:
            st = path_with_fixed_bias(s, fields[:, w, :], opts, xbars[w])
            E, Nn = local_energy(s, st.G)
            out.append((st.logw, st.alive, E, Nn, None))
    return out


def _weighted(rows, mask):
    lw = np.array([r[0].real for r in rows])
    E = np.array([r[2].real for r in rows])
    Nn = np.array([r[3].real for r in rows])
    ref = np.max(lw[mask])
    w = np.where(mask, np.exp(lw - ref), 0.0)
    return np.sum(w * Nn) / np.sum(w), np.sum(w * E) / np.sum(w)


def mu_derivative_fd(sys: UEG, fields, opts: Options = None, h=1e-4, frozen_bias=True):
    """Central finite difference of the phaseless estimates <N> and <E> at
    tau = beta with respect to mu, on the same draws x (Computational
    Details: the interacting mu is tuned so that <N> = N-bar).

    frozen_bias=True holds every slice's force bias at its value on the path
    at mu (the derivative the library accumulates); False lets it follow
    mu.  Walkers killed at mu - h, mu or mu + h but not at all three (a
    cos theta = 0 crossing inside the stencil) are excluded; the count is
    returned.  Returns dict(dN, dE, N, E, excluded)."""
    opts = opts or Options()
    base = mu_observables(sys, fields, opts)
    xb = [r[4] for r in base] if frozen_bias else None
    plus = mu_observables(sys, fields, opts, mu=sys.mu + h, xbars=xb)
    minus = mu_observables(sys, fields, opts, mu=sys.mu - h, xbars=xb)
    a0 = np.array([r[1] for r in base])
    ap = np.array([r[1] for r in plus])
    am = np.array([r[1] for r in minus])
    mask = a0 & ap & am
    excluded = int(np.sum(a0 != mask))
    Np, Ep = _weighted(plus, mask)
    Nm, Em = _weighted(minus, mask)
    N0, E0 = _weighted(base, mask)
    return dict(dN=(Np - Nm) / (2 * h), dE=(Ep - Em) / (2 * h), N=N0, E=E0, excluded=excluded, mask=mask)


def mu_derivative_walkers_fd(sys: UEG, fields, opts: Options = None, h=1e-4):
    """Per-walker central differences in mu at fixed draws and frozen force
    bias: (d ln|w|, d E_L, d N_L, alive at mu-h, mu and mu+h) for every walker."""
    opts = opts or Options()
    base = mu_observables(sys, fields, opts)
    xb = [r[4] for r in base]
    plus = mu_observables(sys, fields, opts, mu=sys.mu + h, xbars=xb)
    minus = mu_observables(sys, fields, opts, mu=sys.mu - h, xbars=xb)
    out = []
    for b, p, m in zip(base, plus, minus):
        ok = b[1] and p[1] and m[1]
        out.append(dict(dlogw=(p[0].real - m[0].real) / (2 * h) if ok else 0.0,
                        dE=(p[2] - m[2]) / (2 * h), dN=(p[3] - m[3]) / (2 * h), alive=ok,
                        logw=b[0].real, E=b[2], N=b[3]))
    return out
