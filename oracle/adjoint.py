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
Both perturbations are rank one, dG = alpha g_k g_k^T with g_k = G e_k (G is symmetric), which
the products below use; the lead broadenings enter through their nonzero boundary blocks.
Pinned by: central finite differences of the direct probe solve (an independent route to T)
and reciprocity of the gradients (dT_RL = dT_LR).
"""
import numpy as np
import scipy.linalg

from . import markov, wire


def _weights_tangent(g, phi, gam, Psi, alpha, col, dgamma):
    """Tangent of every table weight and of the mode weights for dG = alpha col col^T.

    Psi [n, 2W] holds psi = G v for the injection vectors v of both leads (columns p*W + m).
    """
    G = g["G"]
    n, L, W = g["n"], g["L"], g["W"]
    gamma = g["gamma"]
    Gam = [g["GamL"], g["GamR"]]
    sls = [slice(0, W), slice((L - 1) * W, L * W)]
    rows = n + 2 * W
    dw = np.zeros((rows, n + 2))
    dG = alpha * np.outer(col, col)
    # site rows: w[i, j] = gamma_j |G_ji|^2 ; lead: (G^dag Gamma_r G)_ii on the boundary slice
    dw[:n, :n] = (dgamma[None, :] * np.abs(G.T) ** 2
                  + gamma[None, :] * 2.0 * np.real(np.conj(G.T) * dG.T))
    for r in range(2):
        sl = sls[r]
        dw[:n, n + r] = 2.0 * np.real(np.einsum("ai,ab,bi->i", G[sl, :].conj(),
                                                Gam[r][sl, sl], dG[sl, :]))
    du = np.zeros((2, W))
    for p in range(2):
        for m in range(W):
            v = np.zeros(n)
            v[sls[p]] = phi[:, m]
            psi = Psi[:, p * W + m]
            vc = col @ v
            dpsi = alpha * col * vc                           # dG v
            row = n + p * W + m
            dw[row, :n] = dgamma * np.abs(psi) ** 2 + gamma * 2.0 * np.real(np.conj(psi) * dpsi)
            for r in range(2):
                sl = sls[r]
                dw[row, n + r] = 2.0 * np.real(np.vdot(psi[sl], Gam[r][sl, sl] @ dpsi[sl]))
            # d<v|A|v> with A = i (G - G^dag) and v real: i (v^T dG v - conj(v^T dG v))
            z = alpha * vc * vc
            du[p, m] = gam[m] * np.real(1j * (z - np.conj(z)))
    return dw, du


def transmission_gradient(onsite, eta, t, E, p, q, lead_model=0, gamma_lead=0.0, sites=None,
                          slice_h=None):
    """T_qp and its exact derivatives dT/dV [L, W] and dT/deta [L, W] (only the flat site
    indices in ``sites`` when given; the others are left at 0)."""
    onsite = np.asarray(onsite, dtype=np.float64)
    L, W = onsite.shape
    n = L * W
    g = wire.green_retarded(E, onsite, eta, t, lead_model, gamma_lead, slice_h)
    phi, _, gam = wire.lead_modes(E, W, t, lead_model, gamma_lead, slice_h)
    tab = markov.transition_weights(g, (phi, gam))
    w = tab["w"]
    rs = w.sum(1)
    live = rs > 0
    P = np.zeros_like(w)
    P[live] = w[live] / rs[live, None]
    Q = P[:n, :n]
    IQ = np.eye(n) - Q
    lu = scipy.linalg.lu_factor(IQ)                 # (I - Q) is factored once
    h = scipy.linalg.lu_solve(lu, P[:n, n + q])
    inj = slice(n + p * W, n + (p + 1) * W)
    u = tab["mode_w"][p]
    v = P[inj, n + q] + P[inj, :n] @ h
    T = float(u @ v)
    G = g["G"]
    V = np.zeros((n, 2 * W))
    V[:W, :W] = phi
    V[(L - 1) * W:, W:] = phi
    Psi = G @ V
    grads = {}
    ks = range(n) if sites is None else sites
    for kind in ("V", "eta"):
        out = np.zeros(n)
        for k in ks:
            dgamma = np.zeros(n)
            if kind == "V":
                alpha = 1.0
            else:
                alpha = -0.5j
                dgamma[k] = 1.0
            dw, du = _weights_tangent(g, phi, gam, Psi, alpha, G[:, k], dgamma)
            drs = dw.sum(1)
            dP = np.zeros_like(w)
            dP[live] = (dw[live] - P[live] * drs[live, None]) / rs[live, None]
            dh = scipy.linalg.lu_solve(lu, dP[:n, :n] @ h + dP[:n, n + q])
            dv = dP[inj, n + q] + dP[inj, :n] @ h + P[inj, :n] @ dh
            out[k] = du[p] @ v + u @ dv
        grads[kind] = out.reshape(L, W)
    return T, grads["V"], grads["eta"]
