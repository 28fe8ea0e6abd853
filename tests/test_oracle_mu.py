"""Pins of the chemical-potential derivative (CPU).

The library accumulates d/dmu at fixed draws x with the force bias held at
its value on the path: every B carries exp(dtau mu), so
d ln det(I + A_k)/dmu = k dtau (M - tr G(tau_k)) and dG(beta)/dmu =
-beta (I - G) G.  The oracle's definition is the central finite difference
of a full rerun at mu +- h (Computational Details: mu is tuned so that
<N> = N-bar); these tests pin that definition to closed forms and to the
formulas above.
"""
import math

import numpy as np

from oracle import afqmc
from oracle.ueg import UEG, fermi_dirac
from synthetic_inputs import gaussian_fields


def test_noninteracting_number_derivative_closed_form():
    """d<N>/dmu = 2 beta sum f(1-f), d<E>/dmu = 2 beta sum eps f(1-f)."""
    s = UEG(2, 7, 1.0, 0.5, 0.05, interacting=False)
    s.mu = s.mu_T + 0.2
    f = gaussian_fields(3, s.n_slices, 2, s.N_alpha)
    d = afqmc.mu_derivative_fd(s, f)
    ff = fermi_dirac(s.eps, s.mu, s.beta)
    assert abs(d["dN"] - 2 * s.beta * np.sum(ff * (1 - ff))) < 1e-7
    assert abs(d["dE"] - 2 * s.beta * np.sum(s.eps * ff * (1 - ff))) < 1e-7


def test_green_derivative_formula():
    """dG(beta)/dmu = -beta (I - G) G with frozen force bias (central FD)."""
    s = UEG(2, 7, 1.0, 0.5, 0.05)
    f = gaussian_fields(4, s.n_slices, 1, s.N_alpha)[:, 0]
    o = afqmc.Options()
    r = afqmc.propagate_walker(s, f, o, record=True)
    h = 1e-5
    Gp = afqmc.path_with_fixed_bias(afqmc._with_mu(s, s.mu + h), f, o, r.xbar_trace).G
    Gm = afqmc.path_with_fixed_bias(afqmc._with_mu(s, s.mu - h), f, o, r.xbar_trace).G
    G = r.G
    dG = -s.beta * (np.eye(s.M) - G) @ G
    assert np.abs((Gp - Gm) / (2 * h) - dG).max() < 1e-7 * max(1, np.abs(dG).max())


def test_weight_derivative_formula():
    """d ln|w|/dmu = sum_k [Re dlnS_k - tan(theta_k) Im dlnS_k] with
    dlnS_k = 2 dtau (k (M - tr G_k) - (k-1)(M - tr G_{k-1})), against the FD."""
    s = UEG(2, 7, 1.0, 0.5, 0.05)
    W = 6
    f = gaussian_fields(5, s.n_slices, W, s.N_alpha)
    o = afqmc.Options()
    fd = afqmc.mu_derivative_walkers_fd(s, f, o)
    for w in range(W):
        st = afqmc.initial_state(s)
        t_prev = 0j
        dlogw = 0.0
        for k in range(1, s.n_slices + 1):
            st, lnS, _, _ = afqmc.slice_step(s, st, f[k - 1, w], k, o)
            t = k * s.dtau * (s.M - np.trace(st.G))
            dlnS = 2 * (t - t_prev)
            if st.alive:
                dlogw += dlnS.real - math.tan(lnS.imag) * dlnS.imag
            t_prev = t
        if fd[w]["alive"]:
            assert abs(dlogw - fd[w]["dlogw"]) < 1e-6 * max(1, abs(dlogw))


def test_frozen_and_full_bias_derivatives_are_close():
    """The force bias's own mu dependence is a small correction (reported)."""
    s = UEG(2, 7, 1.0, 0.5, 0.05)
    f = gaussian_fields(3, s.n_slices, 16, s.N_alpha)
    a = afqmc.mu_derivative_fd(s, f, frozen_bias=True)
    b = afqmc.mu_derivative_fd(s, f, frozen_bias=False)
    assert abs(a["dN"] - b["dN"]) < 1e-2 * abs(b["dN"])
    assert abs(a["dE"] - b["dE"]) < 1e-2 * abs(b["dE"])
