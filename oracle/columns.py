"""Selected Step 6' table rows of long wires from sparse LU column solves (oracle; test
infrastructure only).

The dense inverse of Eq. eq_for_gr is out of reach for wires of 10^4 - 10^5 sites, but one table
row needs only one column of G^r.  With M = E - H - Sigma^r (Eq. sigmas_comp_r; M is sparse:
nearest-neighbour H, diagonal Sigma_s, the W x W lead blocks on the boundary slices) and its LU
factors (a library primitive), a row's state |v> (a site |i>, or a lead eigenvector |phi_m> on
the boundary slice) gives psi = G |v> = M^{-1} |v>, and the weights of markov.transition_weights
follow: w[v, j] = gamma_j |psi_j|^2 (Eq. draw_i_simult, G symmetric), w[v, lead r] =
<psi|Gamma_r|psi> on the boundary block, <v|A|v> = -2 Im <v|G|v> (v real).
Pinned by: equality with the dense transition_weights on small wires.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import wire


def system_matrix(E, onsite, eta, t, lead_model=0, gamma_lead=0.0):
    """Sparse M = E - H - Sigma_L - Sigma_R - Sigma_s (CSC), and the lead blocks."""
    onsite = np.asarray(onsite, dtype=np.float64)
    L, W = onsite.shape
    n = L * W
    gamma = np.asarray(eta, dtype=np.float64).reshape(n)
    idx = np.arange(n)
    rows, cols, vals = [idx], [idx], [E - onsite.reshape(n) + 0.5j * gamma]
    across = idx[(idx % W) + 1 < W]                      # (k, a) -- (k, a + 1)
    along = idx[idx + W < n]                             # (k, a) -- (k + 1, a)
    for a, b in ((across, across + 1), (along, along + W)):
        rows += [a, b]
        cols += [b, a]
        vals += [np.full(a.size, t, dtype=np.complex128)] * 2   # -H_ij = +t
    phi, sig, gam = wire.lead_modes(E, W, t, lead_model, gamma_lead)
    s_blk = phi @ np.diag(sig) @ phi.T
    g_blk = phi @ np.diag(gam) @ phi.T
    bi, bj = np.meshgrid(np.arange(W), np.arange(W), indexing="ij")
    for k in (0, L - 1):
        rows.append((k * W + bi).ravel())
        cols.append((k * W + bj).ravel())
        vals.append(-s_blk.ravel())
    M = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    return M, phi, gam, g_blk, gamma


def sampled_rows(E, onsite, eta, t, rows, lead_model=0, gamma_lead=0.0):
    """Weights [len(rows), n + 2] and <v|A|v> [len(rows)] of the given table rows (row numbering
    of markov.transition_weights: sites, then the W modes of lead L, then of lead R), plus the
    mode weights [2, W] and c_p [2]."""
    onsite = np.asarray(onsite, dtype=np.float64)
    L, W = onsite.shape
    n = L * W
    M, phi, gam, g_blk, gamma = system_matrix(E, onsite, eta, t, lead_model, gamma_lead)
    lu = spla.splu(M)
    rows = np.asarray(rows, dtype=np.int64)
    V = np.zeros((n, rows.size + 2 * W), dtype=np.complex128)
    for c, r in enumerate(rows):                          # the rows' states
        if r < n:
            V[r, c] = 1.0
        else:
            p, m = divmod(int(r) - n, W)
            k = 0 if p == 0 else L - 1
            V[k * W:(k + 1) * W, c] = phi[:, m]
    for p, k in enumerate((0, L - 1)):                    # every mode (mode weights, c_p)
        V[k * W:(k + 1) * W, rows.size + p * W:rows.size + (p + 1) * W] = phi
    Psi = lu.solve(V)
    sls = [slice(0, W), slice((L - 1) * W, L * W)]
    w = np.zeros((rows.size, n + 2))
    A = np.zeros(rows.size)
    for c in range(rows.size):
        psi = Psi[:, c]
        w[c, :n] = gamma * np.abs(psi) ** 2
        for r_ in range(2):
            sl = sls[r_]
            w[c, n + r_] = np.real(np.vdot(psi[sl], g_blk @ psi[sl]))
        A[c] = -2.0 * np.imag(np.real(V[:, c]) @ psi)
    mode_w = np.zeros((2, W))
    for p in range(2):
        sl = sls[p]
        for m in range(W):
            psi = Psi[:, rows.size + p * W + m]
            mode_w[p, m] = gam[m] * (-2.0 * np.imag(phi[:, m] @ psi[sl]))
    return dict(w=w, A_row=A, mode_w=mode_w, c=mode_w.sum(1))
