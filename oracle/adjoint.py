"""Exact FP64 derivatives of the transmission w.r.t. onsite energies and dephasing
(oracle; test infrastructure only).

The paper does not differentiate its estimator; the derivative target here is the
expectation the walk estimates, T_qp = c_p P(q|p) = sum_m u_m v_m with u_m = lambda_m <phi_m|A|phi_m>
(Eq. lead_out_probability) and v_m the absorption probability at q after injection in mode m
(the absorbing chain of Step 6').  Forward mode, one parameter at a time, exact in FP64:

  dM/dV_k = -e_k e_k^T    =>  dG = G e_k e_k^T G          (M = E - H - Sigma, G = M^{-1})
  dM/deta_k = (i/2) e_k e_k^T  =>  dG = -(i/2) G e_k e_k^T G,  and gamma_k itself moves by 1;
  weights w_ab, row sums, the transition probabilities P_ab = w_ab / rowsum_a, the absorption
  vector h = (I - Q)^{-1} R_q (dh = (I - Q)^{-1} (dQ h + dR_q)), mode weights u_m, and finally
  dT = sum_m du_m v_m + sum_m u_m dv_m.
Pinned by: central finite differences of the direct probe solve (an independent route to T)
and reciprocity of the gradients (dT_RL = dT_LR).
"""
import numpy as np

from . import markov, wire


def _weights_tangent(g, phi, gam, dG, dgamma):
    """Tangent of every table weight, of the row sums and of the mode weights."""
    G = g["G"]
    n, L, W = g["n"], g["L"], g["W"]
    gamma = g["gamma"]
    Gam = [g["GamL"], g["GamR"]]
    Gd = G.conj().T
    dGd = dG.conj().T
    rows = n + 2 * W
    dw = np.zeros((rows, n + 2))
    # site rows: w[i, j] = gamma_j |G_ji|^2, lead: (G^dag Gamma_r G)_ii
    dw[:n, :n] = (dgamma[None, :] * np.abs(G.T) ** 2
                  + gamma[None, :] * 2.0 * np.real(np.conj(G.T) * dG.T))
    for r in range(2):
        dw[:n, n + r] = 2.0 * np.real(np.diag(Gd @ Gam[r] @ dG))
    du = np.zeros((2, W))
    for p, k in enumerate((0, L - 1)):
        for m in range(W):
            v = np.zeros(n, dtype=np.complex128)
            v[k * W:(k + 1) * W] = phi[:, m]
            psi = G @ v
            dpsi = dG @ v
            row = n + p * W + m
            dw[row, :n] = dgamma * np.abs(psi) ** 2 + gamma * 2.0 * np.real(np.conj(psi) * dpsi)
            for r in range(2):
                dw[row, n + r] = 2.0 * np.real(np.vdot(psi, Gam[r] @ dpsi))
            dA = np.real(np.vdot(v, 1j * (dG - dGd) @ v))
            du[p, m] = gam[m] * dA
    return dw, du


def transmission_gradient(onsite, eta, t, E, p, q, lead_model=0, gamma_lead=0.0):
    """T_qp and its exact derivatives dT/dV [L, W] and dT/deta [L, W]."""
    onsite = np.asarray(onsite, dtype=np.float64)
    L, W = onsite.shape
    n = L * W
    g = wire.green_retarded(E, onsite, eta, t, lead_model, gamma_lead)
    phi, _, gam = wire.lead_modes(E, W, t, lead_model, gamma_lead)
    tab = markov.transition_weights(g, (phi, gam))
    w = tab["w"]
    rs = w.sum(1)
    live = rs > 0
    P = np.zeros_like(w)
    P[live] = w[live] / rs[live, None]
    Q = P[:n, :n]
    IQ = np.eye(n) - Q
    h = np.linalg.solve(IQ, P[:n, n + q])
    inj = slice(n + p * W, n + (p + 1) * W)
    u = tab["mode_w"][p]
    v = P[inj, n + q] + P[inj, :n] @ h
    T = float(u @ v)
    G = g["G"]
    grads = {}
    for kind in ("V", "eta"):
        out = np.zeros(n)
        for k in range(n):
            outer = np.outer(G[:, k], G[k, :])
            if kind == "V":
                dG = outer
                dgamma = np.zeros(n)
            else:
                dG = -0.5j * outer
                dgamma = np.zeros(n)
                dgamma[k] = 1.0
            dw, du = _weights_tangent(g, phi, gam, dG, dgamma)
            drs = dw.sum(1)
            dP = np.zeros_like(w)
            dP[live] = (dw[live] - P[live] * drs[live, None]) / rs[live, None]
            dh = np.linalg.solve(IQ, dP[:n, :n] @ h + dP[:n, n + q])
            dv = dP[inj, n + q] + dP[inj, :n] @ h + P[inj, :n] @ dh
            out[k] = du[p] @ v + u @ dv
        grads[kind] = out.reshape(L, W)
    return T, grads["V"], grads["eta"]
