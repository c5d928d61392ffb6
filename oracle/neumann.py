"""The paper's Neumann series for the transmission, summed term by term (oracle; test only).

Eq. (iqof_t_el_db):  T_qp(E) = sum_{n>=0} Tr[Gamma_q Xi^n A_p],  A_p = G Gamma_p G^dag
(Eq. ap_defined), Xi X = G Lambda(X) G^dag (Eq. elastic_xi_op).  In the elastic Buttiker
approximation (Eq. buttiker_scattering_sigma with lambda_i linear in <i|X|i>)
Lambda(X) = sum_i lt_i X_ii |i><i| and charge conservation (Eq. condition4_buttiker, elastic
form) fixes lt_i = gamma_i / A_ii.

Only diagonals propagate: with d^(0) = diag(A_p) and d^(n)_j = sum_i |G_ji|^2 lt_i d^(n-1)_i,
    term_0 = Tr[Gamma_q A_p],   term_n = sum_i lt_i d^(n-1)_i (G^dag Gamma_q G)_ii  (n >= 1).
This is an independent route to T^eff (the Appendix B identity makes it equal to the probe
solve and to the walk's absorption probability); it is used only as a pin.

Pinned by: agreement with the probe solve and the exact chain on wires and chains of several
sizes (test_three_routes_agree), each of those routes pinned by closed forms of its own.
"""
import numpy as np


def neumann_transmission(g, q, p, rtol=1e-14, max_terms=200000):
    G = g["G"]
    gamma = g["gamma"]
    Gam = [g["GamL"], g["GamR"]]
    Gd = G.conj().T
    A_diag = -2.0 * np.imag(np.diag(G))
    lt = np.where(gamma > 0, gamma / A_diag, 0.0)
    Ap = G @ Gam[p] @ Gd
    total = float(np.real(np.trace(Gam[q] @ Ap)))
    d = np.real(np.diag(Ap)).copy()
    out_q = np.real(np.diag(Gd @ Gam[q] @ G))
    absG2 = np.abs(G) ** 2
    prev = None
    for _ in range(max_terms):
        s = lt * d
        term = float(s @ out_q)
        total += term
        # geometric tail estimate term * rho / (1 - rho) from the ratio of successive terms
        if prev is not None and prev > 0.0:
            rho = term / prev
            tail = term * rho / (1.0 - rho) if rho < 1.0 else np.inf
            if tail <= rtol * abs(total):
                break
        elif term == 0.0:
            break
        prev = term
        d = absG2 @ s
    else:
        raise RuntimeError("Neumann series did not converge")
    return total
