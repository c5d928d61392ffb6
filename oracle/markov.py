"""Step 6' transition weights, Step 4 injection and the exact absorbing-chain expectation
(oracle; test infrastructure only).

Table layout (shared contract with the GPU path, stated here so the oracle reads on its own):
rows 0..n-1 are site states |i>; rows n + p*W + m are the injection states |phi_m> of lead p
(p = 0 for L, 1 for R); columns 0..n-1 are sites, column n is lead L and n+1 is lead R.

* Site row i (Sec. II.F, Eq. draw_i_simult and the lead probability of Step 6'):
  with psi = G|i>,   w[i, j] = gamma_j |<j|psi>|^2 = gamma_j |G_ji|^2,
                     w[i, n+r] = <psi|Gamma_r|psi> = (G^dag Gamma_r G)_ii.
* Injection row for eigenvector phi_m of Gamma_p (Sec. II.D Steps 3-5): psi = G|phi_m>, same
  weights.  Each row sums to <i|A|i> (Sec. II.D: sum_b <psi|Gamma_b|psi> + S_n = <i|A|i>).
* Injection distribution (Eq. lead_out_probability): u_m = lambda_m <phi_m|A|phi_m> / Tr[Gamma_p A]
  with A = i (G - G^dag).  c_p = Tr[Gamma_p A] is the estimator value (Eq. elast_lin_xpq).
* Exact expectation of the walk: Q = w[:, :n] / rowsum, R = w[:, n:] / rowsum; absorption
  probabilities from a site are (I - Q)^{-1} R; the mean number of transition draws (steps,
  absorbing draw included, injection draw not) is (I - Q)^{-1} 1.
"""
import numpy as np


def transition_weights(g, lead_model_modes):
    """All table rows' FP64 weights for one task.

    ``lead_model_modes`` = (phi [W, W], gam [W]) eigen-decomposition of Gamma_L = Gamma_R on the
    boundary slice (both leads are identical strips).  Returns dict with
    w [n + 2W, n + 2], mode_w [2, W] (lambda_m <phi_m|A|phi_m>), c [2] (Tr Gamma_p A) and
    A_diag [n + 2W] (<i|A|i> per row, computed from A directly for the row-sum pin).
    """
    G = g["G"]
    n, L, W = g["n"], g["L"], g["W"]
    gamma = g["gamma"]
    Gam = [g["GamL"], g["GamR"]]
    # Gamma_L and Gamma_R vanish outside their boundary slices: every product with them is
    # taken on those W x W blocks
    sls = [slice(0, W), slice((L - 1) * W, L * W)]
    phi, gam = lead_model_modes
    K = n + 2
    rows = n + 2 * W
    w = np.zeros((rows, K))
    A_row = np.zeros(rows)
    # site rows
    absG2 = np.abs(G) ** 2
    w[:n, :n] = absG2.T * gamma[None, :]            # w[i, j] = gamma_j |G_ji|^2
    for r in range(2):
        # (G^dag Gamma_r G)_ii, summed over the boundary slice where Gamma_r is nonzero
        sl = slice((0 if r == 0 else L - 1) * W, (1 if r == 0 else L) * W)
        Gs = G[sl, :]
        w[:n, n + r] = np.real(np.einsum("ai,ab,bi->i", Gs.conj(), Gam[r][sl, sl], Gs))
    A_row[:n] = -2.0 * np.imag(np.diag(G))          # <i|A|i> with A = i (G - G^dag)
    # injection rows and mode distributions
    mode_w = np.zeros((2, W))
    c = np.zeros(2)
    for p, k in enumerate((0, L - 1)):
        sk = sls[p]                                 # phi_m lives on slice k = 0 or L - 1
        A_kk = 1j * (G[sk, sk] - G[sk, sk].conj().T)
        Psi = G[:, sk] @ phi                        # psi_m = G |phi_m>, all modes
        for m in range(W):
            psi = Psi[:, m]
            row = n + p * W + m
            w[row, :n] = gamma * np.abs(psi) ** 2
            for r in range(2):
                sl = sls[r]
                w[row, n + r] = np.real(np.vdot(psi[sl], Gam[r][sl, sl] @ psi[sl]))
            A_row[row] = np.real(np.vdot(phi[:, m], A_kk @ phi[:, m]))
            mode_w[p, m] = gam[m] * A_row[row]
        c[p] = np.real(np.trace(Gam[p][sk, sk] @ A_kk))
    return dict(w=w, mode_w=mode_w, c=c, A_row=A_row, n=n, W=W, K=K)


def absorption(tab):
    """Exact absorption probabilities and mean steps of the Step 6' chain.

    Returns P_site [n, 2], steps_site [n], P_inj [2, 2] (start lead p -> absorbing lead q,
    averaged over the injection distribution), steps_inj [2], steps2_inj [2] (second moment of
    the number of steps) and T_eff [q, p] = c_p P(q|p).  The second moment uses the standard
    absorbing-chain identity E[S_i^2] = ((2N - I) t)_i with N = (I - Q)^{-1}, t = N 1.
    Pinned by: equality with the Buttiker probe solve and the Neumann series; P(L)+P(R) = 1;
    the step moments against brute-force iteration of the chain and the walker's samples.
    """
    w, n, W = tab["w"], tab["n"], tab["W"]
    tot = w.sum(axis=1)
    live = tot > 0
    P = np.zeros_like(w)
    P[live] = w[live] / tot[live, None]
    Q = P[:n, :n]
    R = P[:n, n:]
    IQ = np.eye(n) - Q
    P_site = np.linalg.solve(IQ, R)
    steps_site = np.linalg.solve(IQ, np.ones(n))
    m2_site = 2.0 * np.linalg.solve(IQ, steps_site) - steps_site    # (2N - I) t
    P_inj = np.zeros((2, 2))
    steps_inj = np.zeros(2)
    steps2_inj = np.zeros(2)
    T_eff = np.zeros((2, 2))
    for p in range(2):
        mw = tab["mode_w"][p]
        if mw.sum() <= 0:
            continue
        u = mw / mw.sum()
        rows = slice(n + p * W, n + (p + 1) * W)
        Pi = P[rows]
        P_inj[p] = u @ (Pi[:, n:] + Pi[:, :n] @ P_site)
        steps_inj[p] = u @ (1.0 + Pi[:, :n] @ steps_site)
        # S = 1 + T_j after a first draw to site j (T = 0 when the first draw is a lead)
        steps2_inj[p] = u @ (1.0 + Pi[:, :n] @ (2.0 * steps_site + m2_site))
        T_eff[:, p] = tab["c"][p] * P_inj[p]
    return dict(P_site=P_site, steps_site=steps_site, m2_site=m2_site, P_inj=P_inj,
                steps_inj=steps_inj, steps2_inj=steps2_inj, T_eff=T_eff)
