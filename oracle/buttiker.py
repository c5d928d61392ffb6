"""Direct floating-probe solve of the elastic Buttiker model (oracle; test infrastructure only).

Sec. III.C, Eq. (buteq): with Buttiker scattering the lesser equation reduces to a linear system
over the probe occupations.  Terminals are the two leads and one probe per site i with
Gamma_i = gamma_i |i><i|.  Multi-terminal transmissions T_ab = Tr[Gamma_a G Gamma_b G^dag]:

    T_ij = gamma_i gamma_j |G_ij|^2,   T_iq = gamma_i (G Gamma_q G^dag)_ii,
    T_qp = Tr[Gamma_q G Gamma_p G^dag].

Each probe carries no net current at each energy, so its occupation x_i obeys
    gamma_i A_ii x_i = sum_j T_ij x_j + sum_p T_ip f_p         (sum_b T_ib = gamma_i A_ii),
which is Eq. (buteq) with i_i = gamma_i A_ii x_i.  Solving with f_p = 1 and the other lead at 0
gives the effective transmission  T^eff_qp = T_qp + sum_i T_qi x_i.
Probes with gamma_i = 0 are not terminals and are dropped.
"""
import numpy as np


def terminal_transmissions(g):
    """T_PP [np, np], T_Pq [np, 2], T_qP [2, np], T_qp [2, 2] for leads (L, R) and probes."""
    G = g["G"]
    gamma = g["gamma"]
    probes = np.nonzero(gamma > 0)[0]
    Gl = [g["GamL"], g["GamR"]]
    Gd = G.conj().T
    absG2 = np.abs(G) ** 2
    T_PP = gamma[probes, None] * gamma[None, probes] * absG2[np.ix_(probes, probes)]
    T_Pq = np.empty((probes.size, 2))
    T_qP = np.empty((2, probes.size))
    T_qp = np.empty((2, 2))
    L, W = g["L"], g["W"]
    sls = [slice(0, W), slice((L - 1) * W, L * W)]     # where Gamma_L, Gamma_R are nonzero
    for q in range(2):
        sq = sls[q]
        Gb = Gl[q][sq, sq]
        # (G Gamma_q G^dag)_ii and (G^dag Gamma_q G)_ii, summed over the boundary slice of q
        T_Pq[:, q] = gamma[probes] * np.real(
            np.einsum("ia,ab,ib->i", G[:, sq], Gb, G[:, sq].conj()))[probes]
        T_qP[q, :] = gamma[probes] * np.real(
            np.einsum("ai,ab,bi->i", G[sq, :].conj(), Gb, G[sq, :]))[probes]
        for p in range(2):
            sp = sls[p]
            # Tr[Gamma_q G Gamma_p G^dag] on the two boundary slices
            T_qp[q, p] = np.real(np.trace(Gb @ G[sq, sp] @ Gl[p][sp, sp] @ G[sq, sp].conj().T))
    return probes, T_PP, T_Pq, T_qP, T_qp


def effective_transmission(g):
    """T^eff[q, p] for leads q, p in (L=0, R=1) from the probe system of Eq. (buteq).

    Pinned by: equality with the Neumann series of Eq. (iqof_t_el_db) and with the exact
    absorbing-chain expectation of the walk; reciprocity T^eff_RL = T^eff_LR; probe current
    conservation; the clean-chain/strip closed forms at gamma = 0.
    """
    probes, T_PP, T_Pq, T_qP, T_qp = terminal_transmissions(g)
    Teff = T_qp.copy()
    if probes.size:
        A = -2.0 * np.imag(np.diag(g["G"]))[probes]
        D = np.diag(g["gamma"][probes] * A) - T_PP
        X = np.linalg.solve(D, T_Pq)              # x_i for f_L = 1 (col 0) and f_R = 1 (col 1)
        Teff += T_qP @ X
    return Teff


def probe_occupations(g, f_leads):
    """Probe occupations x_i for given lead occupations (f_L, f_R); used for the
    current-conservation pin (every probe's net current is zero)."""
    probes, T_PP, T_Pq, T_qP, T_qp = terminal_transmissions(g)
    A = -2.0 * np.imag(np.diag(g["G"]))[probes]
    D = np.diag(g["gamma"][probes] * A) - T_PP
    x = np.linalg.solve(D, T_Pq @ np.asarray(f_leads, dtype=np.float64))
    return probes, x, (T_PP, T_Pq, T_qP, T_qp)
