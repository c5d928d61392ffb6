"""Lead current from per-energy transmissions and walk tallies (oracle; test only).

Eq. (iqof_t_el_db): i_q(E) = (1/h) sum_p T_qp(E) (f_p(E) - f_q(E)); with e = h = 1 the current
from lead p to lead q on an energy grid with quadrature weights w_E (midpoint rule of
Sec. III.C) is I = sum_E w_E (f_p(E) - f_q(E)) T_qp(E).

Monte Carlo (Eq. elast_lin_xpq and the binomial variance model of Sec. IV.B.2): every walker
contributes X = c_p delta_{rq}, so with n_q of N walkers absorbed at q,
    T_qp = c_p n_q / N,   SE(T_qp) = c_p sqrt(P (1 - P) / N),  P = n_q / N,
and SE(I)^2 = sum_E (w_E (f_p - f_q))^2 SE(T_qp(E))^2 (energies are sampled independently).

Pinned by: the Fermi function against its closed form and the current against a hand-summed
two-energy case (test_fermi_and_current); the binomial standard error against the spread of
independent replicas (test_binomial_standard_error_is_honest).
"""
import numpy as np


def fermi(E, mu, kT):
    x = (np.asarray(E, dtype=np.float64) - mu) / kT
    return 0.5 * (1.0 - np.tanh(0.5 * x))      # = 1 / (1 + exp(x)), overflow-free


def mc_transmission(c_p, n_q, N):
    c_p = np.asarray(c_p, dtype=np.float64)
    n_q = np.asarray(n_q, dtype=np.float64)
    N = np.asarray(N, dtype=np.float64)
    P = np.where(N > 0, n_q / np.maximum(N, 1), 0.0)
    T = c_p * P
    se = c_p * np.sqrt(np.where(N > 0, P * (1.0 - P) / np.maximum(N, 1), 0.0))
    return T, se


def current(E, w_E, T, se, mu_p, mu_q, kT):
    df = fermi(E, mu_p, kT) - fermi(E, mu_q, kT)
    wd = np.asarray(w_E, dtype=np.float64) * df
    I = float(np.sum(wd * T))
    dI = float(np.sqrt(np.sum((wd * se) ** 2)))
    return I, dI
